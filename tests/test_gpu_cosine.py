"""Parity of the grouped cosine transform (ANOVA_BASIS_COS, the half-period
cosine system of Sec. 5) with the FP64 cosine oracle (oracle/ndct.py).

Bars as for the exponential system: FP32 within 1e-5 relative l2 on the whole
vectors, on every coefficient block of the adjoint and on the forward of each
order class alone; FP64 plans within 1e-6 at the 8 x 8-tap window; LSQR
within 1e-4 of the oracle's LSQR at the same iteration count.
"""
import numpy as np
import pytest

from oracle import ndct, solvers
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


def _layout(terms, bw):
    lens = ndct.block_sizes(terms, bw)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    return offs, lens


def _cos_pair_check(gft, x, terms, bw, tol=TOL, seed=1, f64=False, **plan_kw):
    import torch
    M = x.shape[1]
    n = ndct.n_coeffs(terms, bw)
    fhat = inputs.complex_normal(seed, 2, n)
    y = inputs.complex_normal(seed, 4, M)
    if f64:
        P = gft.Plan(to_dev(x, torch.float64), terms, bw, precision=gft.PREC_F64, basis=gft.BASIS_COS, **plan_kw)
        xo = np.asarray(x, dtype=np.float64)
        cd = torch.complex128
    else:
        P = gft.Plan(to_dev(x, torch.float32), terms, bw, basis=gft.BASIS_COS, **plan_kw)
        xo = f32_nodes(x)
        cd = torch.complex64
    assert P.n_coeffs == n
    f = host(P.trafo(cplx_dev(fhat, cd)))
    g = host(P.adjoint(cplx_dev(y, cd)))
    f_ref = ndct.trafo(xo, terms, bw, fhat)
    g_ref = ndct.adjoint(xo, terms, bw, y)
    assert rel_l2(f, f_ref) <= tol, f"forward {rel_l2(f, f_ref):.3e}"
    assert rel_l2(g, g_ref) <= tol, f"adjoint {rel_l2(g, g_ref):.3e}"
    offs, lens = _layout(terms, bw)
    for u, (o, ln) in enumerate(zip(offs, lens)):
        e = rel_l2(g[o:o + ln], g_ref[o:o + ln])
        assert e <= tol, f"adjoint block {terms[u]}: {e:.3e}"
    for s in sorted({len(u) for u in terms}):
        part = np.zeros_like(fhat)
        for u, (o, ln) in enumerate(zip(offs, lens)):
            if len(terms[u]) == s:
                part[o:o + ln] = fhat[o:o + ln]
        fs = host(P.trafo(cplx_dev(part, cd)))
        e = rel_l2(fs, ndct.trafo(xo, terms, bw, part))
        assert e <= tol, f"forward of the order-{s} terms alone: {e:.3e}"
    return P


@pytest.mark.parametrize("cell_kernel", [0, 1])
def test_cosine_orders_one_to_three(gft, cell_kernel):
    d = 4
    x = inputs.uniform_points(51, d, 4099) + 0.5        # [0, 1)^4
    terms = inputs.terms_up_to(d, 3)
    bw = inputs.bandwidths_by_order(terms, {1: 23, 2: 9, 3: 5})   # odd bandwidths are allowed
    _cos_pair_check(gft, x, terms, bw, cell_kernel=cell_kernel)


def test_cosine_unsorted_spread_and_boundary_nodes(gft):
    d = 3
    x = inputs.uniform_points(52, d, 2000) + 0.5
    x[:, :40] = 0.0          # the cube's faces: phi_k(0) = sqrt 2, phi_k(1) = sqrt 2 (-1)^k
    x[:, 40:80] = 1.0
    x[0, 80:120] = 2.0 - x[0, 120:160]   # outside [0, 1]: the even 2-periodic extension
    terms = inputs.terms_up_to(d, 2)
    bw = inputs.bandwidths_by_order(terms, {1: 16, 2: 12})
    _cos_pair_check(gft, x, terms, bw, node_sort=-1)
    _cos_pair_check(gft, x, terms, bw)


def test_cosine_application_shape(gft):
    """d = 12, |u| <= 2, N = 82 / 10 (6 319 coefficients): the shape of the
    application of Sec. 5, on 5 000 of its 36 160 nodes."""
    w = inputs.cosine_workload(M=5000)
    _cos_pair_check(gft, w["x"], w["terms"], w["bandwidths"])


def test_cosine_fp64_plan(gft):
    d = 3
    x = inputs.uniform_points(53, d, 1500) + 0.5
    terms = inputs.terms_up_to(d, 3)
    # 3-D cosine N = 4 runs at the doubled N = 8 (n = 16): within the FP64 FFT limit n <= 18
    bw = inputs.bandwidths_by_order(terms, {1: 20, 2: 8, 3: 4})
    _cos_pair_check(gft, x, terms, bw, tol=1e-6, f64=True, eps=1e-7)


def test_cosine_lsqr_matches_oracle(gft):
    """Tikhonov LSQR (eq. (new_min_prob)) on a cosine plan (d = 6, |u| <= 2,
    N = 20 / 8, 3 000 uniform nodes in [0, 1]^6, 1 + 6 19 + 15 49 = 850
    unknowns, lambda = 0.1, 15 iterations) against the oracle's LSQR on the
    dense cosine matrix.  (Categorical attributes with few levels, as in the
    application's shape, make most of their columns collinear; that
    rank-deficient case is left to the transform parity tests.)"""
    import torch
    d, M = 6, 3000
    x = inputs.uniform_points(54, d, M) + 0.5
    terms = inputs.terms_up_to(d, 2)
    bw = inputs.bandwidths_by_order(terms, {1: 20, 2: 8})
    y = (inputs.gaussian_bump_sum(x - 0.5, [(0, 1), (3,)]) + 0.01 * inputs.normal(54, 3, M)).astype(np.complex128)
    Phi = ndct.matrix(f32_nodes(x), terms, bw)
    n = Phi.shape[1]
    assert n == 850
    ref = solvers.tikhonov_lsqr(lambda f: Phi @ f, lambda r: Phi.conj().T @ r, y, n, 0.1, None, iters=15)
    P = gft.Plan(to_dev(x, torch.float32), terms, bw, basis=gft.BASIS_COS)
    fh, info, rc = P.lsqr(cplx_dev(y), 0.1, max_it=15)
    assert rc == 0 and info["iterations"] == 15
    assert rel_l2(host(fh), ref.x) <= 1e-4


def test_cosine_rejects_what_the_grids_cannot_hold(gft):
    import torch
    x = torch.rand((2, 100), device="cuda")
    with pytest.raises(gft.AnovaError) as e:
        gft.Plan(x, [(), (0, 1)], [0, 40], basis=gft.BASIS_COS)   # doubled bandwidth 80: grid above 100 KB
    assert e.value.status == -2
