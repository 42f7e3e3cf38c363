"""Parity of the device-driven LSQR and FISTA with the FP64 oracle.

Bar (the benchmark spec): solutions within 1e-4 relative l2 of the oracle and the same
active group set.  The oracle runs the same algorithm with the same iteration
count (LSQR) or to convergence (FISTA, constant step with the same L), on the
same FP32-rounded nodes, with exact dense products.
"""
import numpy as np
import pytest

from oracle import anova, ndft, solvers
from paper_2010_10199_gb300 import inputs

from gpu_util import cplx_dev, f32_nodes, host, rel_l2, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def gft():
    from paper_2010_10199_gb300 import build, gft as g
    build.build()
    g.load()
    return g


def _dense_ops(x, terms, bw):
    Fm = ndft.matrix(f32_nodes(x), terms, bw)
    return Fm, (lambda f: Fm @ f), (lambda r: Fm.conj().T @ r)


def _plan(gft, x, terms, bw, eps=0.0):
    import torch
    return gft.Plan(to_dev(x, torch.float32), terms, bw, eps=eps)


def test_lsqr_c1_fixed_iterations(gft):
    """The small configuration: lambda = 1e-3, 50 iterations."""
    w = inputs.c1_small()
    x, terms, bw, y = w["x"], w["terms"], w["bandwidths"], w["y"]
    n = anova.n_coeffs(terms, bw)
    Fm, F, FH = _dense_ops(x, terms, bw)
    ref = solvers.tikhonov_lsqr(F, FH, y, n, w["lam"], None, iters=w["iters"])
    P = _plan(gft, x, terms, bw)
    fh, info, rc = P.lsqr(cplx_dev(y), w["lam"], max_it=w["iters"])
    assert rc == 0 and info["iterations"] == w["iters"]
    assert rel_l2(host(fh), ref.x) <= TOL
    assert abs(info["rnorm"] - ref.rnorm) <= 1e-4 * ref.rnorm   # sqrt(||r||^2 + 2 lam ||f||^2) estimate


def test_lsqr_third_order_workload_shape(gft):
    """LSQR on the shape of the d = 10, |u| <= 3 workload (176 terms, N =
    100 / 24x24 / 10x10x10, 112 276 unknowns, Beta(2,2) nodes) at 3000 nodes:
    a fixed iteration count against the oracle's LSQR on the direct FP64 sums."""
    w = inputs.c3_lsqr(M=3000)
    x, terms, bw, y = w["x"], w["terms"], w["bandwidths"], w["y"]
    n = anova.n_coeffs(terms, bw)
    assert n == 112276
    xo = f32_nodes(x)
    F = lambda f: ndft.trafo(xo, terms, bw, f)
    FH = lambda r: ndft.adjoint(xo, terms, bw, r)
    lam, iters = 0.1, 20
    ref = solvers.tikhonov_lsqr(F, FH, y, n, lam, None, iters=iters)
    P = _plan(gft, x, terms, bw)
    fh, info, rc = P.lsqr(cplx_dev(y), lam, max_it=iters)
    assert rc == 0 and info["iterations"] == iters
    assert rel_l2(host(fh), ref.x) <= TOL
    assert abs(info["rnorm"] - ref.rnorm) <= 1e-4 * ref.rnorm


def test_lsqr_converged_matches_normal_equations(gft):
    w = inputs.c1_small()
    x, terms, bw, y = w["x"], w["terms"], w["bandwidths"], w["y"]
    Fm, F, FH = _dense_ops(x, terms, bw)
    wts = np.array([np.prod([(1 + abs(k)) ** 1.0 for k in row if k != 0]) for row in anova.frequencies(terms, bw, 6)])
    for lam, ww in ((1e-3, None), (1e-2, wts)):
        ref = solvers.tikhonov_direct(Fm, y, lam, ww)
        P = _plan(gft, x, terms, bw, eps=1e-7)   # 8 x 8 taps: operator error ~1e-7
        import torch
        wd = None if ww is None else torch.from_numpy(ww).cuda()
        fh, info, rc = P.lsqr(cplx_dev(y), lam, max_it=400, atol=1e-7, btol=1e-7, w=wd)
        assert rc == 0
        assert rel_l2(host(fh), ref) <= TOL, (lam, info)


def test_lsqr_tensor_grid_closed_form(gft):
    L, d = 8, 3
    g = np.arange(L) / L - 0.5
    X = np.stack([a.reshape(-1) for a in np.meshgrid(g, g, g, indexing="ij")])
    terms = anova.term_set(d, 2)
    bw = [0, 8, 8, 8, 4, 4, 4]
    M = X.shape[1]
    y = inputs.complex_normal(5, 4, M)
    lam = 0.7
    ref = ndft.adjoint(X, terms, bw, y) / (M + 2 * lam)
    P = _plan(gft, X, terms, bw)
    fh, info, rc = P.lsqr(cplx_dev(y), lam, max_it=3)
    assert rel_l2(host(fh), ref) <= TOL


def test_lsqr_breakdown_reports_status(gft):
    # one unknown: exact after one step; the solver stops with a breakdown status
    x = inputs.uniform_points(5, 1, 40)
    P = _plan(gft, x, [()], [0])
    fh, info, rc = P.lsqr(cplx_dev(np.full(40, 2.0 + 1.0j)), 0.0, max_it=10)
    assert abs(host(fh)[0] - (2.0 + 1.0j)) < 1e-5
    assert info["iterations"] <= 2


def _lasso_problem(seed=21, M=400):
    x = inputs.uniform_points(seed, 4, M)
    terms = anova.term_set(4, 2)
    bw = [0] + [8] * 4 + [4] * 6
    y = (np.exp(-8 * x[0] ** 2) * np.exp(-8 * x[1] ** 2) + 0.5 * np.exp(-8 * x[3] ** 2)
         + 0.01 * inputs.normal(seed, 3, M)).astype(np.complex128)
    return x, terms, bw, y


@pytest.mark.parametrize("weighted", [False, True])
def test_fista_path_matches_oracle(gft, weighted):
    x, terms, bw, y = _lasso_problem()
    n = anova.n_coeffs(terms, bw)
    offs, lens = anova.layout(terms, bw)
    Fm, F, FH = _dense_ops(x, terms, bw)
    ww = None
    if weighted:
        K = anova.frequencies(terms, bw, 4)
        ww = np.array([np.prod([(1 + abs(k)) ** 0.5 for k in row if k != 0]) for row in K])
    L = 1.01 * float(np.linalg.norm(Fm, 2) ** 2)
    lams = [8.0, 2.0, 0.5]
    ref = solvers.fista_path(F, FH, y, n, lams, offs, lens, ww, L=L, max_it=20000, tol=1e-10)
    import torch
    P = _plan(gft, x, terms, bw)
    wd = None if ww is None else torch.from_numpy(ww).cuda()
    path, infos, rc = P.fista(cplx_dev(y), lams, max_it=20000, tol=1e-9, L0=L, w=wd)
    assert rc == 0
    for i, (lam, r) in enumerate(ref):
        got = host(path[i])
        act_ref = solvers.group_norms(r.f, offs, lens) > 0
        act = solvers.group_norms(got, offs, lens) > 0
        assert np.array_equal(act, act_ref), (lam, np.nonzero(act ^ act_ref))
        assert rel_l2(got, r.f) <= TOL, (lam, rel_l2(got, r.f))
        assert infos[i]["active_groups"] == int(act_ref.sum())


def test_fista_backtracking_reaches_the_minimiser(gft):
    x, terms, bw, y = _lasso_problem(seed=22)
    offs, lens = anova.layout(terms, bw)
    Fm, F, FH = _dense_ops(x, terms, bw)
    lam = 2.0
    ref = solvers.block_coordinate_group_lasso(Fm, y, lam, offs, lens)
    P = _plan(gft, x, terms, bw)
    path, infos, rc = P.fista(cplx_dev(y), [lam], max_it=6000, tol=1e-9, step_mode=1, L0=1.0, eta=2.0)
    assert rc == 0 and infos[0]["L"] > 1.0
    assert rel_l2(host(path[0]), ref) <= 1e-3


def test_fista_power_iteration_step(gft):
    x, terms, bw, y = _lasso_problem(seed=23)
    offs, lens = anova.layout(terms, bw)
    Fm, F, FH = _dense_ops(x, terms, bw)
    P = _plan(gft, x, terms, bw)
    path, infos, rc = P.fista(cplx_dev(y), [1.0], max_it=20000, tol=1e-9)   # L from power iteration
    # L = 1.08 x the Lanczos estimate of ||F||^2 (a safe upper bound; the
    # estimate is exact here, where the Krylov space runs out)
    assert 1.0 <= infos[0]["L"] / np.linalg.norm(Fm, 2) ** 2 <= 1.09
    ref = solvers.block_coordinate_group_lasso(Fm, y, 1.0, offs, lens)
    assert rel_l2(host(path[0]), ref) <= TOL


def test_kkt_check_on_device(gft):
    x, terms, bw, y = _lasso_problem(seed=24)
    offs, lens = anova.layout(terms, bw)
    Fm, F, FH = _dense_ops(x, terms, bw)
    lam = 2.0
    f = solvers.block_coordinate_group_lasso(Fm, y, lam, offs, lens)
    P = _plan(gft, x, terms, bw)
    viol, nv = P.kkt(cplx_dev(y), cplx_dev(f), lam, rtol=1e-3)
    ref_viol, ref_bad = solvers.kkt_violations(FH(y - F(f)), f, lam, offs, lens, rtol=1e-3)
    assert nv == 0 and ref_bad == []
    assert np.allclose(viol, ref_viol, atol=5e-4)
    f2 = f.copy()
    f2[offs[2]:offs[2] + lens[2]] += 0.05
    viol2, nv2 = P.kkt(cplx_dev(y), cplx_dev(f2), lam, rtol=1e-3)
    assert nv2 >= 1 and viol2[2] > 1e-3


def test_fista_group_mask_equals_reduced_problem(gft):
    x, terms, bw, y = _lasso_problem(seed=25)
    n = anova.n_coeffs(terms, bw)
    offs, lens = anova.layout(terms, bw)
    mask = np.ones(len(terms), dtype=bool)
    mask[[2, 6, 7]] = False
    keep_t = [t for t, m in zip(terms, mask) if m]
    keep_b = [b for b, m in zip(bw, mask) if m]
    Fm_r, F_r, FH_r = _dense_ops(x, keep_t, keep_b)
    o_r, l_r = anova.layout(keep_t, keep_b)
    lam = 1.0
    ref_r = solvers.block_coordinate_group_lasso(Fm_r, y, lam, o_r, l_r)
    P = _plan(gft, x, terms, bw)
    path, infos, rc = P.fista(cplx_dev(y), [lam], max_it=20000, tol=1e-9, group_mask=list(mask))
    got = host(path[0])
    for u in np.nonzero(~mask)[0]:
        assert np.all(got[offs[u]:offs[u] + lens[u]] == 0)
    got_r = np.concatenate([got[offs[u]:offs[u] + lens[u]] for u in np.nonzero(mask)[0]])
    assert rel_l2(got_r, ref_r) <= TOL
