"""Many problems in one launch: the batched transforms and LSQR against the
single-problem path and the FP64 oracle (the many-problem workload: d in 5..15,
|u| <= 2, N = 32 / 16, uneven M)."""
import numpy as np
import pytest

from oracle import ndft, solvers
from paper_2010_10199_gb300 import inputs

from gpu_util import cplx_dev, f32_nodes, host, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gft():
    from paper_2010_10199_gb300 import build, gft as g
    build.build()
    g.load()
    return g


def _problems(n, scale):
    return [inputs.c5_problem(p, scale) for p in range(n)]


def test_batched_transforms_match_oracle_and_single_plans(gft):
    import torch
    probs = _problems(6, 0.05)   # M from a few hundred to ~10^4
    B = gft.Batch([to_dev(w["x"], torch.float32) for w in probs], [w["terms"] for w in probs],
                  [w["bandwidths"] for w in probs])
    fh = [inputs.decaying_coefficients(7 + i, w["terms"], w["bandwidths"]) for i, w in enumerate(probs)]
    ys = [inputs.complex_normal(7 + i, 4, w["M"]) for i, w in enumerate(probs)]
    f_all = host(B.trafo(cplx_dev(np.concatenate(fh))))
    g_all = host(B.adjoint(cplx_dev(np.concatenate(ys))))
    for p, w in enumerate(probs):
        f = f_all[B.node_off[p]:B.node_off[p + 1]]
        g = g_all[B.coef_off[p]:B.coef_off[p + 1]]
        xo = f32_nodes(w["x"])
        assert rel_l2(f, ndft.trafo(xo, w["terms"], w["bandwidths"], fh[p])) <= 1e-5, p
        assert rel_l2(g, ndft.adjoint(xo, w["terms"], w["bandwidths"], ys[p])) <= 1e-5, p
        P1 = gft.Plan(to_dev(w["x"], torch.float32), w["terms"], w["bandwidths"])
        assert rel_l2(f, host(P1.trafo(cplx_dev(fh[p])))) <= 1e-6
        assert rel_l2(g, host(P1.adjoint(cplx_dev(ys[p])))) <= 1e-6


def test_batched_lsqr_matches_oracle(gft):
    import torch
    probs = _problems(5, 0.03)
    B = gft.Batch([to_dev(w["x"], torch.float32) for w in probs], [w["terms"] for w in probs],
                  [w["bandwidths"] for w in probs])
    y_all = np.concatenate([w["y"] for w in probs])
    fh_all, infos, rc = B.lsqr(cplx_dev(y_all), 1e-3, max_it=30)
    fh_all = host(fh_all)
    for p, w in enumerate(probs):
        xo = f32_nodes(w["x"])
        Fm = ndft.matrix(xo, w["terms"], w["bandwidths"])
        n = Fm.shape[1]
        ref = solvers.tikhonov_lsqr(lambda f: Fm @ f, lambda r: Fm.conj().T @ r, w["y"], n, 1e-3, None, iters=30)
        got = fh_all[B.coef_off[p]:B.coef_off[p + 1]]
        assert infos[p]["iterations"] == ref.iterations == 30
        assert rel_l2(got, ref.x) <= 1e-4, (p, rel_l2(got, ref.x))


def test_batched_lsqr_per_problem_stopping(gft):
    # a problem that is solved exactly after one step stops early; the others go on
    import torch
    probs = _problems(3, 0.02)
    x1 = inputs.uniform_points(99, 2, 300)
    probs.insert(1, dict(x=x1, terms=[(), (0,)], bandwidths=[0, 2], y=np.full(300, 1.5 + 0j), M=300))
    B = gft.Batch([to_dev(w["x"], torch.float32) for w in probs], [w["terms"] for w in probs],
                  [w["bandwidths"] for w in probs])
    y_all = np.concatenate([w["y"] for w in probs])
    fh_all, infos, rc = B.lsqr(cplx_dev(y_all), 0.0, max_it=20)
    assert infos[1]["iterations"] < 20 and infos[0]["iterations"] == 20
    got = host(fh_all)[B.coef_off[1]:B.coef_off[2]]
    assert abs(got[0] - 1.5) < 1e-4
