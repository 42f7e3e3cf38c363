"""FP64 solvers around the grouped transform (oracle; test infrastructure only).

Operators are passed in as callables ``A(v)`` / ``AH(u)`` (normally the direct
summations of ``oracle.ndft``) or as a dense matrix, so every step below is
the algorithm as written, on exact (FP64) matrix-vector products.

* Tikhonov problem   min 1/2 ||y - F f||^2 + lam f^H W f          -- eq. (new_min_prob), Sec. 4.1
  Reading: the regulariser carries no factor 1/2, so the normal equations are
  (F^H F + 2 lam W) f = F^H y, and with g = W^{1/2} f the problem is LSQR's
  damped least squares for A = F W^{-1/2} with damp = sqrt(2 lam).
* LSQR               Paige and Saunders (1982), the solver named in Sec. 4.1
* group lasso        min 1/2 ||y - F f||^2 + lam sum_u ||f_u||_{W_u}  -- eq. (alligatoah), Sec. 4.2
* prox p_L           eq. (projection); closed form per group by Theorem
                     (projection) with xi from the root-finding Remark (bisection,
                     then Newton)
* FISTA              Algorithm "FISTA for group lasso" (backtracking), and the
                     constant-step variant of the Remark after it
* KKT                stationarity x - y + lam W x / ||x||_W = 0 from the proof of
                     Lemma (ii), and the zero threshold of Lemma (iii)
* Sobol index        rho(u) = sigma^2(f_u) / sigma^2(f), eq. (gsi), via Parseval on
                     the coefficient blocks; the active set of eq. (activeset)
* L2 error           eq. (L2error) through Parseval's identity
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _vdot(a, b) -> complex:
    return complex(np.vdot(a, b))


def _norm(a) -> float:
    return float(np.sqrt(np.sum(a.real ** 2 + a.imag ** 2)))


# ---------------------------------------------------------------------------
# LSQR
# ---------------------------------------------------------------------------

@dataclass
class LsqrResult:
    x: np.ndarray
    iterations: int
    istop: int
    rnorm: float       # estimate of sqrt(||b - A x||^2 + damp^2 ||x||^2)
    arnorm: float      # estimate of ||A^H r - damp^2 x||
    anorm: float
    history: list = field(default_factory=list)


def lsqr(A, AH, b, n: int, damp: float = 0.0, iters: int = 50,
         atol: float = 0.0, btol: float = 0.0) -> LsqrResult:
    """Paige--Saunders LSQR for min ||A x - b||^2 + damp^2 ||x||^2 from x_0 = 0.

    Golub--Kahan bidiagonalisation (beta u = b - ..., alpha v = A^H u - beta v),
    an extra plane rotation that eliminates the damping row, then the QR update
    of the bidiagonal system.  For complex A all of alpha, beta, rho, c, s, phi
    are real.  Runs ``iters`` iterations unless a breakdown (alpha = 0 or
    beta = 0: the Krylov space is exhausted and x is exact) or the atol/btol
    tests stop it first.
    """
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros(n, dtype=np.complex128)
    beta = _norm(b)
    u = b / beta if beta > 0 else b.copy()
    v = AH(u) if beta > 0 else np.zeros(n, dtype=np.complex128)
    alpha = _norm(v)
    if alpha > 0:
        v = v / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    anorm2 = 0.0
    bnorm = beta
    res = LsqrResult(x, 0, 0, beta, alpha * beta, 0.0)
    if alpha == 0 or beta == 0:
        res.istop = 0
        return res
    xnorm = 0.0
    res2 = 0.0   # sum of psi_k^2: the damping part of the residual estimate
    for it in range(1, iters + 1):
        # bidiagonalisation
        u = A(v) - alpha * u
        beta = _norm(u)
        if beta > 0:
            u = u / beta
        anorm2 += alpha ** 2 + beta ** 2 + damp ** 2
        v_new = AH(u) - beta * v
        alpha_new = _norm(v_new)
        if alpha_new > 0:
            v_new = v_new / alpha_new
        # eliminate the damping term
        rhohat = math.hypot(rhobar, damp)
        c1 = rhobar / rhohat
        s1 = damp / rhohat
        psi = s1 * phibar
        phibar = c1 * phibar
        # plane rotation on the bidiagonal
        rho = math.hypot(rhohat, beta)
        c = rhohat / rho
        s = beta / rho
        theta = s * alpha_new
        rhobar = -c * alpha_new
        phi = c * phibar
        phibar = s * phibar
        # update x and w
        x = x + (phi / rho) * w
        w = v_new - (theta / rho) * w
        v, alpha = v_new, alpha_new
        xnorm = _norm(x)
        res2 += psi * psi
        rnorm = math.sqrt(res2 + phibar * phibar)
        arnorm = alpha * abs(s * phi)
        res = LsqrResult(x, it, 0, rnorm, arnorm, math.sqrt(anorm2))
        res.history.append((rnorm, arnorm))
        if beta == 0 or alpha == 0:
            res.istop = 1
            break
        if btol > 0 and rnorm <= btol * bnorm + atol * math.sqrt(anorm2) * xnorm:
            res.istop = 2
            break
        if atol > 0 and arnorm <= atol * math.sqrt(anorm2) * rnorm:
            res.istop = 3
            break
    res.x = x
    return res


def tikhonov_lsqr(F, FH, y, n: int, lam: float, w=None, iters: int = 50,
                  atol: float = 0.0, btol: float = 0.0):
    """Minimiser of eq. (new_min_prob) by LSQR on A = F W^{-1/2}, damp = sqrt(2 lam)."""
    if w is None:
        ws = np.ones(n)
    else:
        ws = 1.0 / np.sqrt(np.asarray(w, dtype=np.float64))
    r = lsqr(lambda g: F(ws * g), lambda r_: ws * FH(r_), y, n, math.sqrt(2.0 * lam), iters, atol, btol)
    r.x = ws * r.x
    return r


def tikhonov_direct(Fmat: np.ndarray, y, lam: float, w=None) -> np.ndarray:
    """Normal equations (F^H F + 2 lam W) f = F^H y of eq. (new_min_prob)."""
    n = Fmat.shape[1]
    W = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    G = Fmat.conj().T @ Fmat + 2.0 * lam * np.diag(W)
    return np.linalg.solve(G, Fmat.conj().T @ np.asarray(y, dtype=np.complex128))


# ---------------------------------------------------------------------------
# group prox (Theorem (projection) and the Remark on finding xi)
# ---------------------------------------------------------------------------

def _t_of_xi(z2w, w, xi):
    # t(xi) = || z / (1/xi + w) ||_W^2 = sum w |z|^2 / (1/xi + w)^2
    return float(np.sum(z2w / (1.0 / xi + w) ** 2))


def _g_of_s(z2w, w, s):
    # t(1/s) = sum w |z|^2 / (s + w)^2
    return float(np.sum(z2w / (s + w) ** 2))


def prox_group(z: np.ndarray, thr: float, w=None, bisect: int = 40, newton: int = 50):
    """Minimiser of 1/2 ||x - z||^2 + thr ||x||_W for one group.

    Zero when ||(z_k / w_k)||_W = sqrt(sum |z_k|^2 / w_k) <= thr (Lemma (iii);
    equality gives zero).  Otherwise x = diag(1 / (1 + xi w)) z with
    t(xi) = thr^2 (Theorem (projection)); xi is bracketed by bisection on [0, 1]
    if t(1) >= thr^2, else by bisection on s = 1/xi in [0, 1], then refined with
    Newton steps (Remark after the Theorem).  Returns (x, xi); xi = inf for 0.
    """
    z = np.asarray(z, dtype=np.complex128)
    w = np.ones(z.size) if w is None else np.asarray(w, dtype=np.float64)
    a2 = z.real ** 2 + z.imag ** 2
    if math.sqrt(float(np.sum(a2 / w))) <= thr:
        return np.zeros_like(z), math.inf
    z2w = w * a2
    lam2 = thr * thr
    if _t_of_xi(z2w, w, 1.0) >= lam2:
        lo, hi = 0.0, 1.0            # t increasing in xi
        for _ in range(bisect):
            mid = 0.5 * (lo + hi)
            if mid > 0 and _t_of_xi(z2w, w, mid) < lam2:
                lo = mid
            else:
                hi = mid
        xi = 0.5 * (lo + hi)
        for _ in range(newton):
            f = _t_of_xi(z2w, w, xi) - lam2
            # d/dxi of w|z|^2 (1/xi + w)^-2 = 2 w|z|^2 (1/xi + w)^-3 / xi^2
            fp = float(np.sum(2.0 * z2w / (1.0 / xi + w) ** 3)) / (xi * xi)
            step = f / fp
            xi_new = min(max(xi - step, 0.5 * xi), 2.0 * xi)
            if abs(xi_new - xi) <= 1e-16 * abs(xi):
                xi = xi_new
                break
            xi = xi_new
    else:
        lo, hi = 0.0, 1.0            # g(s) = t(1/s) decreasing in s
        for _ in range(bisect):
            mid = 0.5 * (lo + hi)
            if _g_of_s(z2w, w, mid) > lam2:
                lo = mid
            else:
                hi = mid
        s = 0.5 * (lo + hi)
        for _ in range(newton):
            f = _g_of_s(z2w, w, s) - lam2
            fp = float(np.sum(-2.0 * z2w / (s + w) ** 3))
            s_new = s - f / fp
            s_new = min(max(s_new, 0.5 * s), 2.0 * s) if s > 0 else max(s_new, 0.0)
            if abs(s_new - s) <= 1e-16 * max(abs(s), 1e-300):
                s = s_new
                break
            s = s_new
        xi = 1.0 / s if s > 0 else math.inf
        if not math.isfinite(xi):
            return np.zeros_like(z), math.inf
    return z / (1.0 + xi * w), xi


def group_soft_threshold(z: np.ndarray, thr: float) -> np.ndarray:
    """Textbook group soft threshold max(0, 1 - thr/||z||) z (the W = I case)."""
    nz = _norm(z)
    if nz <= thr:
        return np.zeros_like(z)
    return (1.0 - thr / nz) * z


def prox(z, thr, offs, lens, w=None):
    """p_L applied blockwise: eq. (projection) separates over the groups."""
    out = np.empty_like(np.asarray(z, dtype=np.complex128))
    for o, n in zip(offs, lens):
        ww = None if w is None else w[o:o + n]
        out[o:o + n], _ = prox_group(z[o:o + n], thr, ww)
    return out


def group_norms(f, offs, lens, w=None) -> np.ndarray:
    """||f_u||_{W_u} per group."""
    out = np.empty(len(offs))
    for i, (o, n) in enumerate(zip(offs, lens)):
        a2 = f[o:o + n].real ** 2 + f[o:o + n].imag ** 2
        out[i] = math.sqrt(float(np.sum(a2 if w is None else a2 * w[o:o + n])))
    return out


def group_lasso_objective(F, y, f, lam, offs, lens, w=None) -> float:
    """1/2 ||y - F f||^2 + lam sum_u ||f_u||_W (eq. (alligatoah))."""
    r = np.asarray(y) - F(f)
    return 0.5 * _norm(r) ** 2 + lam * float(np.sum(group_norms(f, offs, lens, w)))


# ---------------------------------------------------------------------------
# FISTA
# ---------------------------------------------------------------------------

@dataclass
class FistaResult:
    f: np.ndarray
    iterations: int
    L: float
    converged: bool
    n_products: int   # number of F applications (an F^H comes with each gradient)


def fista(F, FH, y, f0, lam: float, offs, lens, w=None, L0: float = 1.0, eta: float = 2.0,
          max_it: int = 500, tol: float = 0.0, constant_step: bool = False) -> FistaResult:
    """Algorithm "FISTA for group lasso" (Sec. 4.2).

    h_1 = f_0, t_1 = 1; for k = 1..K: L_k = L_{k-1}; f_k = p_{L_k}(h_k);
    while ||y - F f_k||^2 - ||y - F h_k||^2 > 2 Re<f_k - h_k, F^H(F h_k - y)>
    + L_k ||f_k - h_k||^2: L_k = eta L_k, f_k = p_{L_k}(h_k);
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2; h_{k+1} = f_k + (t_k - 1)/t_{k+1} (f_k - f_{k-1}).
    With ``constant_step`` the while loop is skipped (Remark after the Algorithm).
    Stops early when ||f_k - f_{k-1}|| <= tol ||f_k||.
    """
    y = np.asarray(y, dtype=np.complex128)
    f_prev = np.array(f0, dtype=np.complex128)
    h = f_prev.copy()
    t = 1.0
    L = L0
    nprod = 0
    converged = False
    k = 0
    for k in range(1, max_it + 1):
        Fh = F(h)
        nprod += 1
        rh = Fh - y
        grad = FH(rh)
        f = prox(h - grad / L, lam / L, offs, lens, w)
        if not constant_step:
            rh2 = _norm(rh) ** 2
            while True:
                rf = F(f) - y
                nprod += 1
                dfh = f - h
                lhs = _norm(rf) ** 2 - rh2
                rhs = 2.0 * _vdot(dfh, grad).real + L * _norm(dfh) ** 2
                if lhs <= rhs:
                    break
                L *= eta
                f = prox(h - grad / L, lam / L, offs, lens, w)
        t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        h = f + ((t - 1.0) / t_next) * (f - f_prev)
        dn = _norm(f - f_prev)
        fn = _norm(f)
        f_prev = f
        t = t_next
        if tol > 0 and dn <= tol * max(fn, 1e-300):
            converged = True
            break
    return FistaResult(f_prev, k, L, converged, nprod)


def power_norm2(F, FH, n: int, iters: int = 30, seed_vec=None) -> float:
    """Estimate of ||F||_2^2 = lambda_max(F^H F) by power iteration from a fixed vector."""
    v = np.ones(n, dtype=np.complex128) if seed_vec is None else np.asarray(seed_vec, dtype=np.complex128)
    v = v / _norm(v)
    lam = 0.0
    for _ in range(iters):
        g = FH(F(v))
        lam = _vdot(v, g).real
        ng = _norm(g)
        if ng == 0:
            return 0.0
        v = g / ng
    return lam


def fista_path(F, FH, y, n: int, lambdas, offs, lens, w=None, L=None, max_it=500, tol=1e-9,
               constant_step=True, eta=2.0):
    """Warm-started lambda path from the largest lambda with f_0 = 0 (experiments of Sec. 4.2)."""
    f = np.zeros(n, dtype=np.complex128)
    out = []
    for lam in sorted(lambdas, reverse=True):
        r = fista(F, FH, y, f, lam, offs, lens, w, L0=L, eta=eta, max_it=max_it, tol=tol,
                  constant_step=constant_step)
        f = r.f
        out.append((lam, r))
    return out


# ---------------------------------------------------------------------------
# optimality checks and sensitivity indices
# ---------------------------------------------------------------------------

def kkt_violations(FH_r: np.ndarray, f: np.ndarray, lam: float, offs, lens, w=None, rtol: float = 1e-6):
    """Group-lasso optimality per group with g = F^H (y - F f):
    inactive u (f_u = 0): ||W^{-1/2} g_u|| <= lam (Lemma (iii));
    active u: g_u = lam W f_u / ||f_u||_W (stationarity in the proof of Lemma (ii)).
    Returns (per-group violation measure, list of violating group ids)."""
    viol = np.zeros(len(offs))
    bad = []
    for i, (o, n) in enumerate(zip(offs, lens)):
        g = FH_r[o:o + n]
        x = f[o:o + n]
        ww = np.ones(n) if w is None else w[o:o + n]
        xn = math.sqrt(float(np.sum(ww * (x.real ** 2 + x.imag ** 2))))
        if xn == 0.0:
            v = math.sqrt(float(np.sum((g.real ** 2 + g.imag ** 2) / ww))) - lam
            viol[i] = v / lam
        else:
            v = _norm(g - lam * ww * x / xn)
            viol[i] = v / lam
        if viol[i] > rtol:
            bad.append(i)
    return viol, bad


def sobol_indices(f: np.ndarray, offs, lens) -> np.ndarray:
    """rho(u) = ||f_u||^2 / sum_{v != empty} ||f_v||^2 (eq. (gsi) with Parseval);
    the empty set gets 0."""
    e = np.array([float(np.sum(np.abs(f[o:o + n]) ** 2)) for o, n in zip(offs, lens)])
    total = float(np.sum(e[1:])) if len(e) > 1 else 0.0
    rho = np.zeros_like(e)
    if total > 0:
        rho[1:] = e[1:] / total
    return rho


def l2_error(fhat: np.ndarray, c: np.ndarray, norm2: float) -> float:
    """Relative L2 error of eq. (L2error) through Parseval's identity:
    ||f - S f||^2 = ||f||^2 + sum_{k in I} |fhat_k - c_k|^2 - sum_{k in I} |c_k|^2,
    with c_k the exact coefficients of f on I and norm2 = ||f||^2; returns
    ||f - S f|| / ||f||."""
    d = np.asarray(fhat, dtype=np.complex128) - np.asarray(c, dtype=np.complex128)
    e2 = norm2 + float(np.sum(d.real ** 2 + d.imag ** 2)) - float(np.sum(np.abs(c) ** 2))
    return math.sqrt(max(e2, 0.0) / norm2)


def active_set(rho: np.ndarray, terms, eps_by_order) -> list:
    """U* = {empty} cup {u : rho(u) > eps_|u|} (eq. (activeset))."""
    return [i for i, u in enumerate(terms) if len(u) == 0 or rho[i] > eps_by_order[len(u) - 1]]


def block_coordinate_group_lasso(Fmat: np.ndarray, y, lam: float, offs, lens, w=None,
                                 sweeps: int = 20000, tol: float = 1e-13) -> np.ndarray:
    """Independent reference minimiser of eq. (alligatoah) for tiny problems:
    cyclic block-coordinate proximal steps, each block with its own Lipschitz
    constant ||F_u||^2, until no block moves by more than ``tol``."""
    y = np.asarray(y, dtype=np.complex128)
    n = Fmat.shape[1]
    f = np.zeros(n, dtype=np.complex128)
    r = y.copy()  # r = y - F f
    Lu = [float(np.linalg.norm(Fmat[:, o:o + m], 2) ** 2) for o, m in zip(offs, lens)]
    for _ in range(sweeps):
        move = 0.0
        for (o, m), L in zip(zip(offs, lens), Lu):
            Fu = Fmat[:, o:o + m]
            old = f[o:o + m].copy()
            z = old + (Fu.conj().T @ r) / L
            new, _ = prox_group(z, lam / L, None if w is None else w[o:o + m])
            delta = new - old
            if np.any(delta != 0):
                r -= Fu @ delta
                f[o:o + m] = new
                move = max(move, _norm(delta))
        if move <= tol:
            break
    return f
