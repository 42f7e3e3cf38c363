"""Pins of the oracle's solvers against closed forms, library routines and an
independent minimiser (none of them reuse the code under test)."""
import math

import numpy as np
import pytest

from oracle import anova, ndft, solvers
from paper_2010_10199_gb300 import inputs


def _grid_problem(L=8, d=3):
    g = np.arange(L) / L - 0.5
    X = np.stack([a.reshape(-1) for a in np.meshgrid(*([g] * d), indexing="ij")])
    terms = anova.term_set(d, 2)
    bw = [0] + [8] * d + [4] * (len(terms) - 1 - d)
    return X, terms, bw


def _ops(x, terms, bw):
    return (lambda f: ndft.trafo(x, terms, bw, f), lambda y: ndft.adjoint(x, terms, bw, y))


# ------------------------------------------------------------------ LSQR ----

def test_lsqr_tensor_grid_closed_form():
    # F^H F = M I on the grid, so the Tikhonov minimiser is F^H y / (M + 2 lam w)
    X, terms, bw = _grid_problem()
    M = X.shape[1]
    n = anova.n_coeffs(terms, bw)
    F, FH = _ops(X, terms, bw)
    y = inputs.complex_normal(1, 4, M)
    # weights with three distinct values: A^H A + damp^2 I has three distinct
    # eigenvalues, so LSQR (a Krylov method) is exact after three iterations
    w = np.array([1.0, 2.5, 4.0])[(inputs.uniform(1, 9, n) * 3).astype(int)]
    for lam in (1e-3, 1.0, 50.0):
        r = solvers.tikhonov_lsqr(F, FH, y, n, lam, w, iters=3)
        ref = FH(y) / (M + 2 * lam * w)
        assert np.linalg.norm(r.x - ref) / np.linalg.norm(ref) < 1e-12
        r1 = solvers.tikhonov_lsqr(F, FH, y, n, lam, None, iters=1)  # w = 1: one step
        ref1 = FH(y) / (M + 2 * lam)
        assert np.linalg.norm(r1.x - ref1) / np.linalg.norm(ref1) < 1e-12


def test_lsqr_matches_normal_equations():
    w_ = inputs.c1_small()
    x, terms, bw = w_["x"][:, :600], w_["terms"], w_["bandwidths"]
    y = w_["y"][:600]
    n = anova.n_coeffs(terms, bw)
    F, FH = _ops(x, terms, bw)
    Fm = ndft.matrix(x, terms, bw)
    wts = 1.0 + inputs.uniform(2, 9, n)
    for lam, w in ((1e-3, None), (1e-1, wts)):
        ref = solvers.tikhonov_direct(Fm, y, lam, w)
        r = solvers.tikhonov_lsqr(F, FH, y, n, lam, w, iters=800, atol=1e-14, btol=1e-14)
        assert np.linalg.norm(r.x - ref) / np.linalg.norm(ref) < 1e-8


def test_lsqr_unregularised_matches_lstsq():
    # M > |I| and full rank: the least-squares problem (min_prob) has a unique solution
    x = inputs.uniform_points(4, 3, 400)
    terms = anova.term_set(3, 2)
    bw = [0, 8, 8, 8, 4, 4, 4]
    n = anova.n_coeffs(terms, bw)
    F, FH = _ops(x, terms, bw)
    Fm = ndft.matrix(x, terms, bw)
    y = inputs.complex_normal(4, 4, 400)
    ref = np.linalg.lstsq(Fm, y, rcond=None)[0]
    r = solvers.lsqr(F, FH, y, n, 0.0, iters=500, atol=1e-15, btol=1e-15)
    assert np.linalg.norm(r.x - ref) / np.linalg.norm(ref) < 1e-9


def test_lsqr_breakdown_exact_solution():
    # one column: the Krylov space is exhausted after one step
    x = inputs.uniform_points(5, 1, 20)
    F, FH = _ops(x, [()], [0])
    r = solvers.lsqr(F, FH, np.full(20, 3.0 + 0j), 1, 0.0, iters=10, atol=1e-12, btol=1e-12)
    assert r.iterations <= 2 and r.istop > 0 and abs(r.x[0] - 3.0) < 1e-13


# ------------------------------------------------------------------ prox ----

def test_prox_unit_weights_is_group_soft_threshold():
    for seed in range(20):
        z = inputs.complex_normal(seed, 2, 7)
        thr = float(inputs.uniform(seed, 3, 1)[0]) * 4.0
        x, _ = solvers.prox_group(z, thr)
        assert np.allclose(x, solvers.group_soft_threshold(z, thr), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("branch", ["xi_below_one", "xi_above_one"])
def test_prox_general_weights_stationarity(branch):
    # x - z + thr W x / ||x||_W = 0 (proof of Lemma (ii)); both bisection branches
    z = inputs.complex_normal(11, 2, 9) * 5.0
    w = 1.0 + inputs.uniform(11, 3, 9) * 9.0
    zero_thr = math.sqrt(float(np.sum(np.abs(z) ** 2 / w)))
    xi1_thr = math.sqrt(float(np.sum(w * np.abs(z) ** 2 / (1.0 + w) ** 2)))  # sqrt(t(1))
    thr = 0.5 * xi1_thr if branch == "xi_below_one" else 0.5 * (xi1_thr + zero_thr)
    x, xi = solvers.prox_group(z, thr, w)
    assert (xi < 1.0) == (branch == "xi_below_one")
    xn = math.sqrt(float(np.sum(w * np.abs(x) ** 2)))
    res = x - z + thr * w * x / xn
    assert np.linalg.norm(res) / np.linalg.norm(z) < 1e-12
    # and it is the minimiser: random perturbations do not decrease the objective
    obj = lambda v: 0.5 * np.linalg.norm(v - z) ** 2 + thr * math.sqrt(float(np.sum(w * np.abs(v) ** 2)))
    base = obj(x)
    for s in range(20):
        p = inputs.complex_normal(100 + s, 2, 9) * 1e-4
        assert obj(x + p) >= base - 1e-12


def test_prox_zero_threshold_boundary():
    # Lemma (iii): zero iff thr >= ||(z_k/w_k)||_W ; equality gives zero
    z = np.array([3.0 + 4.0j, 0.0, 1.0j])
    w = np.array([1.0, 2.0, 4.0])
    t0 = math.sqrt(float(np.sum(np.abs(z) ** 2 / w)))
    x, _ = solvers.prox_group(z, t0, w)
    assert np.all(x == 0)
    x, _ = solvers.prox_group(z, t0 * (1 - 1e-6), w)
    assert np.any(x != 0)


# ----------------------------------------------------------------- FISTA ----

def test_fista_tensor_grid_closed_form():
    # separable on the grid: with L = M the prox step is exact after one iteration
    X, terms, bw = _grid_problem()
    M = X.shape[1]
    n = anova.n_coeffs(terms, bw)
    offs, lens = anova.layout(terms, bw)
    F, FH = _ops(X, terms, bw)
    y = inputs.complex_normal(2, 4, M)
    z = FH(y) / M
    gn = solvers.group_norms(z, offs, lens)
    lam = float(np.median(gn)) * M  # about half the groups survive
    ref = np.concatenate([max(0.0, 1.0 - lam / (M * gn[i])) * z[o:o + m]
                          for i, (o, m) in enumerate(zip(offs, lens))])
    r = solvers.fista(F, FH, y, np.zeros(n), lam, offs, lens, L0=float(M), max_it=30,
                      constant_step=True, tol=1e-15)
    assert np.linalg.norm(r.f - ref) / np.linalg.norm(ref) < 1e-12
    assert 0 < np.count_nonzero(solvers.group_norms(r.f, offs, lens)) < len(offs)


def _tiny_lasso():
    x = inputs.uniform_points(21, 3, 60)
    terms = anova.term_set(3, 2)
    bw = [0, 4, 4, 4, 4, 2, 4]
    n = anova.n_coeffs(terms, bw)
    offs, lens = anova.layout(terms, bw)
    Fm = ndft.matrix(x, terms, bw)  # dense operator: same products, far less call overhead
    F, FH = (lambda f: Fm @ f), (lambda r: Fm.conj().T @ r)
    y = (np.exp(-8 * x[0] ** 2) * np.exp(-8 * x[1] ** 2)).astype(np.complex128)
    return x, terms, bw, n, offs, lens, F, FH, y


def test_fista_matches_block_coordinate_minimiser():
    x, terms, bw, n, offs, lens, F, FH, y = _tiny_lasso()
    assert n <= 50
    Fm = ndft.matrix(x, terms, bw)
    L = 1.01 * float(np.linalg.norm(Fm, 2) ** 2)
    w = 1.0 + inputs.uniform(3, 9, n)
    for lam, ww in ((2.0, None), (0.5, w)):
        ref = solvers.block_coordinate_group_lasso(Fm, y, lam, offs, lens, ww)
        r = solvers.fista(F, FH, y, np.zeros(n), lam, offs, lens, ww, L0=L, max_it=20000,
                          constant_step=True, tol=1e-14)
        assert np.linalg.norm(r.f - ref) / max(np.linalg.norm(ref), 1e-12) < 1e-6
        act_ref = solvers.group_norms(ref, offs, lens) > 0
        act = solvers.group_norms(r.f, offs, lens) > 0
        assert np.array_equal(act, act_ref)


def test_fista_backtracking_reaches_same_minimiser():
    x, terms, bw, n, offs, lens, F, FH, y = _tiny_lasso()
    lam = 1.0
    Lc = 1.01 * solvers.power_norm2(F, FH, n, iters=200)
    a = solvers.fista(F, FH, y, np.zeros(n), lam, offs, lens, L0=Lc, max_it=20000,
                      constant_step=True, tol=1e-14)
    b = solvers.fista(F, FH, y, np.zeros(n), lam, offs, lens, L0=1.0, eta=2.0, max_it=6000,
                      constant_step=False, tol=1e-14)
    assert b.L >= 1.0 and b.n_products > b.iterations
    Fm = ndft.matrix(x, terms, bw)
    ref = solvers.block_coordinate_group_lasso(Fm, y, lam, offs, lens)
    assert np.linalg.norm(a.f - ref) / np.linalg.norm(ref) < 1e-6
    assert np.linalg.norm(b.f - ref) / np.linalg.norm(ref) < 1e-5


def test_kkt_holds_at_minimiser_and_fails_elsewhere():
    x, terms, bw, n, offs, lens, F, FH, y = _tiny_lasso()
    Fm = ndft.matrix(x, terms, bw)
    lam = 1.5
    f = solvers.block_coordinate_group_lasso(Fm, y, lam, offs, lens)
    g = FH(y - F(f))
    viol, bad = solvers.kkt_violations(g, f, lam, offs, lens, rtol=1e-6)
    assert bad == []
    f2 = f.copy()
    f2[offs[1]:offs[1] + lens[1]] += 0.05
    g2 = FH(y - F(f2))
    _, bad2 = solvers.kkt_violations(g2, f2, lam, offs, lens, rtol=1e-6)
    assert 1 in bad2


def test_power_iteration_matches_svd():
    x, terms, bw, n, offs, lens, F, FH, y = _tiny_lasso()
    Fm = ndft.matrix(x, terms, bw)
    est = solvers.power_norm2(F, FH, n, iters=300)
    assert abs(est - np.linalg.norm(Fm, 2) ** 2) / est < 1e-8


def _sobol_pins_hold(sobol) -> bool:
    """Values of rho(u) = sigma^2(f_u) / sigma^2(f) (eq. (gsi)) worked out by
    hand through Parseval: sigma^2(f_u) = sum_{k in block u} |c_k|^2 and
    sigma^2(f) = ||f||^2 - |c_0|^2 = the sum over the non-empty blocks."""
    ok = True
    # blocks: empty {c_0 = 100}, u1 {2}, u2 {1}: energies 4 and 1 -> 4/5, 1/5;
    # c_0 is the mean and does not enter the variance
    f = np.array([100.0, 2.0, 1.0], dtype=np.complex128)
    rho = sobol(f, np.array([0, 1, 2]), np.array([1, 1, 1]))
    ok &= bool(np.allclose(rho, [0.0, 0.8, 0.2], rtol=0, atol=1e-15))
    # several coefficients per block, complex values: |1+1j|^2 + |1|^2 = 3,
    # |2j|^2 + |-1|^2 + |0|^2 = 5, |3|^2 = 9 -> 3/17, 5/17, 9/17
    f = np.array([7 - 3j, 1 + 1j, 1, 2j, -1, 0, 3], dtype=np.complex128)
    rho = sobol(f, np.array([0, 1, 3, 6]), np.array([1, 2, 3, 1]))
    ok &= bool(np.allclose(rho, [0.0, 3 / 17, 5 / 17, 9 / 17], rtol=0, atol=1e-15))
    return ok


def test_sobol_indices_match_hand_values():
    assert _sobol_pins_hold(solvers.sobol_indices)


def test_sobol_pins_catch_planted_mistakes():
    """Each plausible mistake in rho(u) fails the hand-worked values above."""
    def no_square(f, offs, lens):       # |c_k| instead of |c_k|^2 (Parseval's square dropped)
        e = np.array([float(np.sum(np.abs(f[o:o + n]))) for o, n in zip(offs, lens)])
        r = np.zeros_like(e)
        r[1:] = e[1:] / e[1:].sum()
        return r

    def with_mean(f, offs, lens):       # ||f||^2 instead of ||f||^2 - |c_0|^2 in the denominator
        e = np.array([float(np.sum(np.abs(f[o:o + n]) ** 2)) for o, n in zip(offs, lens)])
        r = e / e.sum()
        r[0] = 0.0
        return r

    def real_only(f, offs, lens):       # Re(c_k)^2 only
        e = np.array([float(np.sum(f[o:o + n].real ** 2)) for o, n in zip(offs, lens)])
        r = np.zeros_like(e)
        r[1:] = e[1:] / e[1:].sum()
        return r

    for bad in (no_square, with_mean, real_only):
        assert not _sobol_pins_hold(bad), bad.__name__


def _active_set_pins_hold(active) -> bool:
    """U* = {empty} cup {u : rho(u) > eps_|u|} (eq. (activeset)): strict
    inequality, the threshold chosen by the order of u, the empty set always in."""
    terms = [(), (0,), (1,), (0, 1), (0, 1, 2), (2,)]
    rho = np.array([0.0, 0.3, 0.1, 0.1, 0.05, 0.1])
    eps = [0.1, 0.05, 0.01]   # eps_1, eps_2, eps_3
    # (0,): 0.3 > 0.1 in; (1,): 0.1 = eps_1 out; (0,1): 0.1 > 0.05 in;
    # (0,1,2): 0.05 > 0.01 in; (2,): 0.1 = eps_1 out; the empty set in although rho = 0
    ok = active(rho, terms, eps) == [0, 1, 3, 4]
    ok &= active(np.zeros(6), terms, eps) == [0]
    return bool(ok)


def test_active_set_matches_hand_values():
    assert _active_set_pins_hold(solvers.active_set)


def test_active_set_pins_catch_planted_mistakes():
    def ge(rho, terms, eps):            # >= instead of >
        return [i for i, u in enumerate(terms) if len(u) == 0 or rho[i] >= eps[len(u) - 1]]

    def no_empty(rho, terms, eps):      # the empty set left out
        return [i for i, u in enumerate(terms) if len(u) > 0 and rho[i] > eps[len(u) - 1]]

    def order_index(rho, terms, eps):   # eps indexed by |u| instead of |u| - 1
        return [i for i, u in enumerate(terms) if len(u) == 0 or rho[i] > eps[min(len(u), len(eps) - 1)]]

    for bad in (ge, no_empty, order_index):
        assert not _active_set_pins_hold(bad), bad.__name__


def test_lsqr_residual_estimate_is_the_damped_residual():
    # Paige--Saunders: rnorm = sqrt(||b - A x||^2 + damp^2 ||x||^2), from the
    # accumulated psi_k^2 and phibar (exact in exact arithmetic)
    w_ = inputs.c1_small()
    x, terms, bw, y = w_["x"][:, :500], w_["terms"], w_["bandwidths"], w_["y"][:500]
    Fm = ndft.matrix(x, terms, bw)
    n = Fm.shape[1]
    for lam, iters in ((1e-3, 7), (0.5, 30)):
        r = solvers.tikhonov_lsqr(lambda f: Fm @ f, lambda q: Fm.conj().T @ q, y, n, lam, None, iters=iters)
        true = math.sqrt(np.linalg.norm(y - Fm @ r.x) ** 2 + 2 * lam * np.linalg.norm(r.x) ** 2)
        assert abs(r.rnorm - true) <= 1e-10 * true
