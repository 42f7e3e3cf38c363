"""Precision study of the grid storage: FP32 grids against FP16 and BF16 grids
with FP32 arithmetic, on the 1e4-node subsample of the d = 20 workload (all
211 terms), each against the FP64 oracle on the same FP32 nodes.

A 16-bit grid value carries a relative rounding error of at most 2^-11 (FP16)
or 2^-8 (BF16); every output sums many rounded values with window weights, so
the relative l2 error of the transforms stays near half that unit.  Bars:
FP32 1e-5 (the path's bar), FP16 1e-3, BF16 8e-3, and the ordering
FP32 < FP16 < BF16.  The solvers run on 16-bit plans unchanged (vectors stay
FP32); LSQR on the small workload reaches the FP16 grid accuracy.
"""
import numpy as np
import pytest

from oracle import anova, ndft, solvers
from paper_2010_10199_gb300 import inputs

from gpu_util import cplx_dev, f32_nodes, host, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gft():
    from paper_2010_10199_gb300 import build, gft as g
    build.build()
    g.load()
    return g


@pytest.fixture(scope="module")
def c2_sub():
    w = inputs.c2_scale(M=10000)
    xo = f32_nodes(w["x"])
    f_ref = ndft.trafo(xo, w["terms"], w["bandwidths"], w["fhat"])
    g_ref = ndft.adjoint(xo, w["terms"], w["bandwidths"], w["y"])
    return w, f_ref, g_ref


def _errors(gft, w, f_ref, g_ref, precision):
    import torch
    P = gft.Plan(to_dev(w["x"], torch.float32), w["terms"], w["bandwidths"], precision=precision)
    f = host(P.trafo(cplx_dev(w["fhat"])))
    g = host(P.adjoint(cplx_dev(w["y"])))
    return rel_l2(f, f_ref), rel_l2(g, g_ref)


def test_grid_precision_study(gft, c2_sub):
    w, f_ref, g_ref = c2_sub
    e32 = _errors(gft, w, f_ref, g_ref, gft.PREC_F32)
    e16 = _errors(gft, w, f_ref, g_ref, gft.PREC_F16)
    eb16 = _errors(gft, w, f_ref, g_ref, gft.PREC_BF16)
    print("relative l2 (forward, adjoint): fp32", e32, "fp16", e16, "bf16", eb16)
    assert max(e32) <= 1e-5
    assert max(e16) <= 1e-3
    assert max(eb16) <= 8e-3
    for k in range(2):
        assert e32[k] < e16[k] < eb16[k]


@pytest.mark.parametrize("precision", ["F16", "BF16"])
def test_16bit_grids_ragged_and_third_order(gft, precision):
    prec = getattr(gft, "PREC_" + precision)
    bar = 1e-3 if precision == "F16" else 8e-3
    import torch
    for x, terms, bw in ((inputs.uniform_points(7, 5, 4099), anova.term_set(5, 2), [0] + [16] * 5 + [8] * 10),
                         (inputs.beta22_points(3, 4, 3000), anova.term_set(4, 3),
                          [0] + [20] * 4 + [12] * 6 + [10] * 4)):
        xo = f32_nodes(x)
        fhat = inputs.decaying_coefficients(1, terms, bw)
        y = inputs.complex_normal(1, 4, x.shape[1])
        P = gft.Plan(to_dev(x, torch.float32), terms, bw, precision=prec)
        assert rel_l2(host(P.trafo(cplx_dev(fhat))), ndft.trafo(xo, terms, bw, fhat)) <= bar
        assert rel_l2(host(P.adjoint(cplx_dev(y))), ndft.adjoint(xo, terms, bw, y)) <= bar


def test_lsqr_on_fp16_grids(gft):
    import torch
    w = inputs.c1_small()
    x, terms, bw, y = w["x"], w["terms"], w["bandwidths"], w["y"]
    n = anova.n_coeffs(terms, bw)
    Fm = ndft.matrix(f32_nodes(x), terms, bw)
    ref = solvers.tikhonov_lsqr(lambda f: Fm @ f, lambda r: Fm.conj().T @ r, y, n, w["lam"], None,
                                iters=w["iters"])
    P = gft.Plan(to_dev(x, torch.float32), terms, bw, precision=gft.PREC_F16)
    fh, info, rc = P.lsqr(cplx_dev(y), w["lam"], max_it=w["iters"])
    assert rc in (0, -5)
    assert rel_l2(host(fh), ref.x) <= 5e-3
