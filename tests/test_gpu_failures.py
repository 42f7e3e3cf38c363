"""Failure paths of the library, made on the host or with benign device inputs.

* Non-finite data: a NaN or an infinity in y reaches the FP64 solver scalars,
  which the solvers report as ANOVA_ERR_NOT_FINITE (no kernel indexes memory
  with a data value, so such inputs cannot fault).
* Out of memory: anova_debug_fail_allocation makes the k-th allocation of a
  plan creation (device or host) fail as an exhausted device or host would.
  Every k either returns ANOVA_ERR_NOMEM with everything freed, or -- for the
  optional allocations (the cell-sorted node copy, the fixed-point
  accumulators) -- a plan without that part whose transforms still meet the
  1e-5 bar against the FP64 oracle.  The free device memory returns to its
  level before the failures.
"""
import numpy as np
import pytest

from oracle import ndft
from paper_2010_10199_gb300 import inputs

from gpu_util import cplx_dev, f32_nodes, host, rel_l2, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def gft():
    import torch
    from paper_2010_10199_gb300 import build, gft as g
    assert torch.cuda.is_available()
    build.build()
    g.load()
    return g


def _small():
    w = inputs.c1_small()
    return w["x"], w["terms"], w["bandwidths"], w["y"]


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_lsqr_reports_non_finite_data(gft, bad):
    import torch
    x, terms, bw, y = _small()
    P = gft.Plan(to_dev(x, torch.float32), terms, bw)
    yb = y.copy()
    yb[17] = bad
    with pytest.raises(gft.AnovaError) as e:
        P.lsqr(cplx_dev(yb), 1e-3, max_it=20)
    assert e.value.status == -7   # ANOVA_ERR_NOT_FINITE
    # the plan stays usable: the same call on finite data succeeds
    fh, info, rc = P.lsqr(cplx_dev(y), 1e-3, max_it=20)
    assert rc == 0 and info["iterations"] == 20 and np.all(np.isfinite(host(fh)))


def test_fista_reports_non_finite_data(gft):
    import torch
    x, terms, bw, y = _small()
    P = gft.Plan(to_dev(x, torch.float32), terms, bw)
    yb = y.copy()
    yb[3] = np.nan
    with pytest.raises(gft.AnovaError) as e:
        P.fista(cplx_dev(yb), [1.0], max_it=50)
    assert e.value.status == -7
    path, infos, rc = P.fista(cplx_dev(y), [1.0], max_it=50)
    assert rc == 0 and np.all(np.isfinite(host(path)))


def test_injected_allocation_failures_free_everything(gft):
    import torch
    x, terms, bw, y = _small()
    xo = f32_nodes(x)
    xd = to_dev(x, torch.float32)
    fhat = inputs.decaying_coefficients(5, terms, bw)
    f_ref = ndft.trafo(xo, terms, bw, fhat)
    g_ref = ndft.adjoint(xo, terms, bw, y)
    fh_d, y_d = cplx_dev(fhat), cplx_dev(y)

    def full_use():
        P = gft.Plan(xd, terms, bw)
        f = host(P.trafo(fh_d))
        g = host(P.adjoint(y_d))
        P.lsqr(y_d, 1e-3, max_it=3)
        P.close()
        return f, g

    full_use()                      # loads every kernel module this test touches
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    outcomes = []
    try:
        for k in range(1, 48):
            gft.anova_debug_fail_allocation(k)
            try:
                P = gft.Plan(xd, terms, bw)
            except gft.AnovaError as e:
                assert e.status == -3, f"k={k}: status {e.status}"   # ANOVA_ERR_NOMEM
                outcomes.append("nomem")
                continue
            finally:
                gft.anova_debug_fail_allocation(0)
            # an optional allocation failed (or none did): the plan must still be right
            f = host(P.trafo(fh_d))
            g = host(P.adjoint(y_d))
            assert rel_l2(f, f_ref) <= TOL and rel_l2(g, g_ref) <= TOL, f"k={k}"
            P.close()
            outcomes.append("ok")
    finally:
        gft.anova_debug_fail_allocation(0)
    assert outcomes.count("nomem") >= 20          # every required allocation was hit
    assert outcomes[-1] == "ok"                   # past the last allocation nothing fails
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 <= (4 << 20), f"device memory lost: {free0 - free1} bytes"


def test_injected_failure_of_the_solver_workspace(gft):
    import torch
    x, terms, bw, y = _small()
    P = gft.Plan(to_dev(x, torch.float32), terms, bw)
    y_d = cplx_dev(y)
    gft.anova_debug_fail_allocation(1)
    try:
        with pytest.raises(gft.AnovaError) as e:
            P.lsqr(y_d, 1e-3, max_it=5)
        assert e.value.status == -3
    finally:
        gft.anova_debug_fail_allocation(0)
    fh, info, rc = P.lsqr(y_d, 1e-3, max_it=5)   # the workspace is created on the next call
    assert rc == 0 and info["iterations"] == 5
