"""ctypes binding of the C ABI in ``include/anova_gft.h`` (argument marshalling only).

Every computation runs in ``libanova_gft.so``; this module converts Python
arguments to the C types and checks status codes.  There is no fallback: if
the shared library is missing or cannot be loaded, every call raises.

The raw entry points keep the C names (``anova_plan_create``, ``grouped_trafo``,
``grouped_adjoint``, ``lsqr_solve``, ``fista_solve``, ...).  ``Plan`` is a small
convenience wrapper that takes torch CUDA tensors and passes their device
pointers and the current stream.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libanova_gft.so")

PREC_F32, PREC_BF16, PREC_F16, PREC_F64 = 0, 1, 2, 3
BASIS_EXP, BASIS_COS = 0, 1

_lib = None


class AnovaError(RuntimeError):
    def __init__(self, fn: str, status: int, text: str):
        super().__init__(f"{fn} failed: {text} ({status})")
        self.status = status


class PlanOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("eps", ctypes.c_double), ("window_m_col", ctypes.c_int),
                ("window_m_row", ctypes.c_int), ("sigma", ctypes.c_double), ("n_ctas", ctypes.c_int),
                ("node_sort", ctypes.c_int), ("cell_kernel", ctypes.c_int), ("basis", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("stop_reason", ctypes.c_int),
                ("n_trafo", ctypes.c_int), ("n_adjoint", ctypes.c_int), ("active_groups", ctypes.c_int),
                ("rnorm", ctypes.c_double), ("arnorm", ctypes.c_double), ("objective", ctypes.c_double),
                ("L", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ScreenStats(ctypes.Structure):
    _fields_ = [("proposed_groups", ctypes.c_int64), ("readmitted_groups", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("term_iterations", ctypes.c_int64), ("full_term_iterations", ctypes.c_int64),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


N_SCREEN_FEATURES = 7


class TuneTrial(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("window_m_row", ctypes.c_int), ("n_ctas", ctypes.c_int),
                ("node_sort", ctypes.c_int), ("cell_kernel", ctypes.c_int), ("ms_pair", ctypes.c_double),
                ("est_error", ctypes.c_double), ("chosen", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def library_path() -> str:
    return LIB_PATH


def load(path: str | None = None):
    """Load libanova_gft.so (raises if it is missing: there is no CPU path)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    vp, i32p, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    lib.anova_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int64, vp, ctypes.c_int,
                                      i32p, i32p, ctypes.POINTER(PlanOptions), vp]
    lib.anova_plan_create.restype = ctypes.c_int
    lib.anova_plan_destroy.argtypes = [vp]
    lib.anova_plan_destroy.restype = None
    lib.anova_num_coeffs.argtypes = [vp]
    lib.anova_num_coeffs.restype = ctypes.c_int64
    lib.anova_term_offset.argtypes = [vp, ctypes.c_int, i64p, i64p]
    lib.anova_term_offset.restype = ctypes.c_int
    lib.anova_term_grid.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]
    lib.anova_term_grid.restype = ctypes.c_int
    lib.grouped_trafo.argtypes = [vp, vp, vp]
    lib.grouped_trafo.restype = ctypes.c_int
    lib.grouped_adjoint.argtypes = [vp, vp, vp]
    lib.grouped_adjoint.restype = ctypes.c_int
    lib.lsqr_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double, vp,
                               ctypes.POINTER(SolveInfo)]
    lib.lsqr_solve.restype = ctypes.c_int
    lib.fista_solve.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.POINTER(ctypes.c_uint8), ctypes.c_int, vp, ctypes.POINTER(SolveInfo)]
    lib.fista_solve.restype = ctypes.c_int
    lib.anova_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.anova_profile_enable.restype = ctypes.c_int
    lib.anova_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_char_p), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.c_int]
    lib.anova_profile_read.restype = ctypes.c_int
    lib.anova_mlp_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, vp, vp]
    lib.anova_mlp_create.restype = ctypes.c_int
    lib.anova_mlp_destroy.argtypes = [vp]
    lib.anova_mlp_destroy.restype = None
    lib.anova_mlp_num_params.argtypes = [vp]
    lib.anova_mlp_num_params.restype = ctypes.c_int64
    lib.anova_mlp_get_params.argtypes = [vp, vp, vp]
    lib.anova_mlp_get_params.restype = ctypes.c_int
    lib.anova_mlp_forward.argtypes = [vp, vp, ctypes.c_int, vp]
    lib.anova_mlp_forward.restype = ctypes.c_int
    lib.anova_mlp_gradients.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
    lib.anova_mlp_gradients.restype = ctypes.c_int
    lib.anova_mlp_train.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                    ctypes.c_float, vp]
    lib.anova_mlp_train.restype = ctypes.c_int
    lib.anova_screen_features.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, vp]
    lib.anova_screen_features.restype = ctypes.c_int
    lib.fista_screened_path.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, vp,
                                        ctypes.POINTER(SolveInfo), ctypes.POINTER(ScreenStats)]
    lib.fista_screened_path.restype = ctypes.c_int
    lib.anova_plan_autotune.argtypes = [ctypes.POINTER(PlanOptions), ctypes.c_int, ctypes.c_int64, vp, ctypes.c_int,
                                        i32p, i32p, ctypes.c_double, ctypes.c_int, ctypes.POINTER(TuneTrial),
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int), vp]
    lib.anova_plan_autotune.restype = ctypes.c_int
    lib.anova_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(i32p), ctypes.POINTER(i32p), ctypes.POINTER(PlanOptions), vp]
    lib.anova_batch_create.restype = ctypes.c_int
    lib.anova_batch_destroy.argtypes = [vp]
    lib.anova_batch_destroy.restype = None
    lib.anova_batch_layout.argtypes = [vp, i64p, i64p]
    lib.anova_batch_layout.restype = ctypes.c_int
    lib.grouped_trafo_batch.argtypes = [vp, vp, vp]
    lib.grouped_trafo_batch.restype = ctypes.c_int
    lib.grouped_adjoint_batch.argtypes = [vp, vp, vp]
    lib.grouped_adjoint_batch.restype = ctypes.c_int
    lib.lsqr_solve_batch.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, vp, ctypes.POINTER(SolveInfo)]
    lib.lsqr_solve_batch.restype = ctypes.c_int
    lib.anova_kkt_check.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    lib.anova_kkt_check.restype = ctypes.c_int
    lib.grouped_trafo_noalloc.argtypes = [ctypes.c_int, ctypes.c_int64, vp, ctypes.c_int, i32p, i32p, vp, vp, vp]
    lib.grouped_trafo_noalloc.restype = ctypes.c_int
    lib.anova_sobol_indices.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_uint8)]
    lib.anova_sobol_indices.restype = ctypes.c_int
    lib.anova_l2_error.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.anova_l2_error.restype = ctypes.c_int
    lib.anova_debug_fail_allocation.argtypes = [ctypes.c_int]
    lib.anova_debug_fail_allocation.restype = ctypes.c_int
    lib.anova_status_string.argtypes = [ctypes.c_int]
    lib.anova_status_string.restype = ctypes.c_char_p
    lib.anova_version.argtypes = []
    lib.anova_version.restype = ctypes.c_char_p
    if path is None:
        _lib = lib
    return lib


def _check(fn: str, rc: int):
    if rc != 0:
        raise AnovaError(fn, rc, load().anova_status_string(rc).decode())
    return rc


# ------------------------------------------------------------ raw C names --

def anova_plan_create(d, M, x_ptr, term_dims, bandwidth, opts: PlanOptions | None = None, stream=0):
    """term_dims: list of tuples (|u| <= 3); bandwidth: list of ints.  Returns the handle."""
    lib = load()
    n = len(term_dims)
    td = (ctypes.c_int32 * (3 * n))()
    bw = (ctypes.c_int32 * n)()
    for i, u in enumerate(term_dims):
        u = tuple(int(c) for c in u)
        if len(u) > 3:
            raise AnovaError("anova_plan_create", -2, "term order above 3")
        for j in range(3):
            td[3 * i + j] = u[j] if j < len(u) else -1
        bw[i] = int(bandwidth[i]) if len(u) else 0
    h = ctypes.c_void_p()
    rc = lib.anova_plan_create(ctypes.byref(h), int(d), int(M), ctypes.c_void_p(int(x_ptr) or None), n, td, bw,
                               ctypes.byref(opts) if opts is not None else None, ctypes.c_void_p(int(stream) or None))
    _check("anova_plan_create", rc)
    return h


def autotune(x, terms, bandwidths, eps: float = 1e-5, reps: int = 3, stream=None):
    """Plan options chosen by anova_plan_autotune for FP32 node tensor x [d, M];
    returns (options dict for Plan(...), list of trial dicts)."""
    import torch
    x = x.to(torch.float32).contiguous()
    d, M = int(x.shape[0]), int(x.shape[1])
    n = len(terms)
    td = (ctypes.c_int32 * (3 * n))()
    bw = (ctypes.c_int32 * n)()
    for i, u in enumerate(terms):
        u = tuple(int(c) for c in u)
        for j in range(3):
            td[3 * i + j] = u[j] if j < len(u) else -1
        bw[i] = int(bandwidths[i]) if len(u) else 0
    opts = PlanOptions(precision=PREC_F32, eps=0.0, window_m_col=0, window_m_row=0, sigma=0.0, n_ctas=0,
                       node_sort=0, cell_kernel=0, basis=BASIS_EXP)
    trials = (TuneTrial * 32)()
    nt = ctypes.c_int(0)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = load().anova_plan_autotune(ctypes.byref(opts), d, M, ctypes.c_void_p(x.data_ptr()), n, td, bw, float(eps),
                                    int(reps), trials, 32, ctypes.byref(nt), ctypes.c_void_p(st.cuda_stream or None))
    _check("anova_plan_autotune", rc)
    chosen = {"sigma": opts.sigma, "window_m_row": opts.window_m_row, "n_ctas": opts.n_ctas,
              "node_sort": opts.node_sort, "cell_kernel": opts.cell_kernel}
    return chosen, [trials[i].as_dict() for i in range(nt.value)]


def anova_plan_destroy(h):
    load().anova_plan_destroy(h)


def anova_num_coeffs(h) -> int:
    return int(load().anova_num_coeffs(h))


def anova_term_offset(h, u):
    off, ln = ctypes.c_int64(), ctypes.c_int64()
    _check("anova_term_offset", load().anova_term_offset(h, int(u), ctypes.byref(off), ctypes.byref(ln)))
    return off.value, ln.value


def anova_term_grid(h, u):
    n, mc, mr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check("anova_term_grid", load().anova_term_grid(h, int(u), ctypes.byref(n), ctypes.byref(mc), ctypes.byref(mr)))
    return n.value, mc.value, mr.value


def grouped_trafo(h, fhat_ptr, f_ptr):
    return _check("grouped_trafo", load().grouped_trafo(h, ctypes.c_void_p(int(fhat_ptr) or None),
                                                        ctypes.c_void_p(int(f_ptr) or None)))


def grouped_adjoint(h, y_ptr, fhat_ptr):
    return _check("grouped_adjoint", load().grouped_adjoint(h, ctypes.c_void_p(int(y_ptr) or None),
                                                            ctypes.c_void_p(int(fhat_ptr) or None)))


def grouped_trafo_noalloc(d, M, x_ptr, term_dims, bandwidth, fhat_ptr, f_ptr, stream=0):
    """Plan-free forward transform whose working memory is a static device array
    (for callers that cannot allocate device memory; see include/anova_gft.h)."""
    n = len(term_dims)
    td = (ctypes.c_int32 * (3 * n))()
    bw = (ctypes.c_int32 * n)()
    for i, u in enumerate(term_dims):
        u = tuple(int(c) for c in u)
        for j in range(3):
            td[3 * i + j] = u[j] if j < len(u) else -1
        bw[i] = int(bandwidth[i]) if len(u) else 0
    rc = load().grouped_trafo_noalloc(int(d), int(M), ctypes.c_void_p(int(x_ptr) or None), n, td, bw,
                                      ctypes.c_void_p(int(fhat_ptr) or None), ctypes.c_void_p(int(f_ptr) or None),
                                      ctypes.c_void_p(int(stream) or None))
    return _check("grouped_trafo_noalloc", rc)


def lsqr_solve(h, y_ptr, w_ptr, lam, max_it, atol, btol, fhat_ptr):
    info = SolveInfo()
    rc = load().lsqr_solve(h, ctypes.c_void_p(int(y_ptr) or None), ctypes.c_void_p(int(w_ptr) or None), float(lam),
                           int(max_it), float(atol), float(btol), ctypes.c_void_p(int(fhat_ptr) or None),
                           ctypes.byref(info))
    if rc not in (0, -5):
        _check("lsqr_solve", rc)
    return rc, info


def fista_solve(h, y_ptr, w_ptr, lambdas, max_it, tol, step_mode, L0, eta, group_mask, warm_start, path_ptr):
    n = len(lambdas)
    lam = (ctypes.c_double * n)(*[float(v) for v in lambdas])
    infos = (SolveInfo * n)()
    mask = None
    if group_mask is not None:
        mask = (ctypes.c_uint8 * len(group_mask))(*[1 if v else 0 for v in group_mask])
    rc = load().fista_solve(h, ctypes.c_void_p(int(y_ptr) or None), ctypes.c_void_p(int(w_ptr) or None), lam, n,
                            int(max_it), float(tol), int(step_mode), float(L0), float(eta), mask, int(warm_start),
                            ctypes.c_void_p(int(path_ptr) or None), infos)
    if rc not in (0, -5):
        _check("fista_solve", rc)
    return rc, [infos[i] for i in range(n)]


def anova_kkt_check(h, y_ptr, w_ptr, fhat_ptr, lam, rtol, n_terms):
    viol = (ctypes.c_double * max(1, n_terms))()
    nv = ctypes.c_int()
    _check("anova_kkt_check", load().anova_kkt_check(h, ctypes.c_void_p(int(y_ptr) or None),
                                                     ctypes.c_void_p(int(w_ptr) or None),
                                                     ctypes.c_void_p(int(fhat_ptr) or None), float(lam), float(rtol),
                                                     viol, ctypes.byref(nv)))
    return [viol[i] for i in range(n_terms)], nv.value


def anova_profile_enable(h, on: bool = True):
    return _check("anova_profile_enable", load().anova_profile_enable(h, 1 if on else 0))


def anova_profile_read(h, reset: bool = False) -> dict:
    """{stage name: (milliseconds, launches)} since the last reset."""
    n = 16
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    names = (ctypes.c_char_p * n)()
    ns = ctypes.c_int()
    _check("anova_profile_read", load().anova_profile_read(h, ms, cnt, names, n, ctypes.byref(ns), 1 if reset else 0))
    return {names[i].decode(): (ms[i], int(cnt[i])) for i in range(min(ns.value, n))}


def anova_sobol_indices(h, fhat_ptr, n_terms, eps_by_order=None):
    """Sobol indices rho(u) (eq. (gsi)) of a coefficient vector and, with
    thresholds (eps_1, eps_2, eps_3), the active-set flags of eq. (activeset)."""
    rho = (ctypes.c_double * max(1, n_terms))()
    eps = (ctypes.c_double * 3)(*[float(v) for v in eps_by_order]) if eps_by_order is not None else None
    act = (ctypes.c_uint8 * max(1, n_terms))() if eps_by_order is not None else None
    _check("anova_sobol_indices", load().anova_sobol_indices(h, ctypes.c_void_p(int(fhat_ptr) or None), rho, eps, act))
    return [rho[i] for i in range(n_terms)], (None if act is None else [bool(act[i]) for i in range(n_terms)])


def anova_l2_error(h, fhat_ptr, c_ptr, norm2):
    """Relative L2 error of eq. (L2error) through Parseval's identity."""
    err = ctypes.c_double()
    _check("anova_l2_error", load().anova_l2_error(h, ctypes.c_void_p(int(fhat_ptr) or None),
                                                   ctypes.c_void_p(int(c_ptr) or None), float(norm2),
                                                   ctypes.byref(err)))
    return err.value


def anova_debug_fail_allocation(k: int):
    """Make the k-th following plan allocation fail (test fault injection; 0 cancels)."""
    return _check("anova_debug_fail_allocation", load().anova_debug_fail_allocation(int(k)))


def anova_status_string(status: int) -> str:
    return load().anova_status_string(int(status)).decode()


def anova_version() -> str:
    return load().anova_version().decode()


# ---------------------------------------------------------- torch helper --

class Plan:
    """Owns an anova plan for torch CUDA node tensor ``x`` of shape [d, M]."""

    def __init__(self, x, terms, bandwidths, precision: int = PREC_F32, eps: float = 0.0, sigma: float = 0.0,
                 window_m_row: int = 0, n_ctas: int = 0, node_sort: int = 0, cell_kernel: int = 0,
                 basis: int = BASIS_EXP, stream=None):
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda):
            raise TypeError("x must be a CUDA tensor [d, M]")
        self.real = torch.float64 if precision == PREC_F64 else torch.float32
        self.cplx = torch.complex128 if precision == PREC_F64 else torch.complex64
        x = x.to(self.real).contiguous()
        self.d, self.M = int(x.shape[0]), int(x.shape[1])
        self.terms = [tuple(u) for u in terms]
        self.bandwidths = [int(b) for b in bandwidths]
        self.basis = int(basis)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        opts = PlanOptions(precision=precision, eps=eps, window_m_col=0, window_m_row=window_m_row, sigma=sigma,
                           n_ctas=n_ctas, node_sort=node_sort, cell_kernel=cell_kernel, basis=basis)
        self.handle = anova_plan_create(self.d, self.M, x.data_ptr() if self.M else 0, self.terms,
                                        self.bandwidths, opts, self.stream.cuda_stream)
        self.n_coeffs = anova_num_coeffs(self.handle)
        self.device = x.device

    def close(self):
        if getattr(self, "handle", None):
            anova_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, v, n, name):
        import torch
        if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == self.cplx and v.numel() == n
                and v.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous CUDA {self.cplx} tensor with {n} entries")
        return v

    def trafo(self, fhat, out=None):
        import torch
        self._vec(fhat, self.n_coeffs, "fhat")
        out = torch.empty(self.M, dtype=self.cplx, device=self.device) if out is None else out
        self._vec(out, self.M, "out")
        grouped_trafo(self.handle, fhat.data_ptr() if self.n_coeffs else 0, out.data_ptr() if self.M else 0)
        return out

    def adjoint(self, y, out=None):
        import torch
        self._vec(y, self.M, "y")
        out = torch.empty(self.n_coeffs, dtype=self.cplx, device=self.device) if out is None else out
        self._vec(out, self.n_coeffs, "out")
        grouped_adjoint(self.handle, y.data_ptr() if self.M else 0, out.data_ptr())
        return out

    def _weights(self, w):
        import torch
        if w is None:
            return 0
        if not (isinstance(w, torch.Tensor) and w.is_cuda and w.dtype == torch.float64 and w.numel() == self.n_coeffs
                and w.is_contiguous()):
            raise TypeError(f"w must be a contiguous CUDA float64 tensor with {self.n_coeffs} entries")
        return w.data_ptr()

    def lsqr(self, y, lam, max_it=50, atol=0.0, btol=0.0, w=None, out=None):
        """Tikhonov minimiser of eq. (new_min_prob) by LSQR; returns (fhat, info dict, status)."""
        import torch
        self._vec(y, self.M, "y")
        out = torch.empty(self.n_coeffs, dtype=self.cplx, device=self.device) if out is None else out
        rc, info = lsqr_solve(self.handle, y.data_ptr() if self.M else 0, self._weights(w), lam, max_it, atol, btol,
                              out.data_ptr())
        return out, info.as_dict(), rc

    def fista(self, y, lambdas, max_it=500, tol=1e-6, step_mode=0, L0=0.0, eta=2.0, w=None, group_mask=None,
              warm_start=None):
        """Group-lasso path of eq. (alligatoah); returns (path [n_lambda, n_coeffs], infos, status)."""
        import torch
        self._vec(y, self.M, "y")
        path = torch.zeros((len(lambdas), self.n_coeffs), dtype=self.cplx, device=self.device)
        if warm_start is not None:
            path[0].copy_(warm_start)
        rc, infos = fista_solve(self.handle, y.data_ptr(), self._weights(w), list(lambdas), max_it, tol, step_mode,
                                L0, eta, group_mask, 1 if warm_start is not None else 0, path.data_ptr())
        return path, [i.as_dict() for i in infos], rc

    def kkt(self, y, fhat, lam, rtol=1e-3, w=None):
        self._vec(y, self.M, "y")
        self._vec(fhat, self.n_coeffs, "fhat")
        return anova_kkt_check(self.handle, y.data_ptr(), self._weights(w), fhat.data_ptr(), lam, rtol,
                               len(self.terms))

    def sobol(self, fhat, eps_by_order=None):
        """Sobol indices of the blocks of fhat (and the active-set flags with thresholds)."""
        self._vec(fhat, self.n_coeffs, "fhat")
        return anova_sobol_indices(self.handle, fhat.data_ptr(), len(self.terms), eps_by_order)

    def l2_error(self, fhat, c, norm2):
        """Relative L2 error of eq. (L2error) for exact coefficients c on this plan's index set."""
        self._vec(fhat, self.n_coeffs, "fhat")
        self._vec(c, self.n_coeffs, "c")
        return anova_l2_error(self.handle, fhat.data_ptr(), c.data_ptr(), norm2)

    def profile(self, on: bool = True):
        anova_profile_enable(self.handle, on)

    def profile_read(self, reset: bool = False) -> dict:
        return anova_profile_read(self.handle, reset)

    def term_offset(self, u):
        return anova_term_offset(self.handle, u)

    def term_grid(self, u):
        return anova_term_grid(self.handle, u)


# ------------------------------------------------------------- screening --

class Mlp:
    """The group-screening network (two hidden ReLU layers, sigmoid output)."""

    def __init__(self, params, n_features: int = N_SCREEN_FEATURES, hidden: int = 128, stream=None):
        import numpy as np
        import torch
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        self.F, self.H = int(n_features), int(hidden)
        expect = self.F * self.H + self.H + self.H * self.H + self.H + self.H + 1
        if p.size != expect:
            raise ValueError(f"expected {expect} parameters, got {p.size}")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check("anova_mlp_create", load().anova_mlp_create(ctypes.byref(h), self.F, self.H,
                                                           ctypes.c_void_p(p.ctypes.data),
                                                           ctypes.c_void_p(self.stream.cuda_stream or None)))
        self.handle = h
        self.n_params = expect

    def close(self):
        if getattr(self, "handle", None):
            load().anova_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self, grads: bool = False):
        import numpy as np
        p = np.empty(self.n_params, dtype=np.float32)
        g = np.empty(self.n_params, dtype=np.float32) if grads else None
        _check("anova_mlp_get_params", load().anova_mlp_get_params(
            self.handle, ctypes.c_void_p(p.ctypes.data), ctypes.c_void_p(g.ctypes.data) if grads else None))
        return (p, g) if grads else p

    def forward(self, X):
        import torch
        G = int(X.shape[0])
        out = torch.empty(G, dtype=torch.float32, device=X.device)
        _check("anova_mlp_forward", load().anova_mlp_forward(self.handle, ctypes.c_void_p(X.data_ptr() or None), G,
                                                             ctypes.c_void_p(out.data_ptr() or None)))
        return out

    def gradients(self, X, y, pos_weight: float = 1.0):
        loss = ctypes.c_double()
        _check("anova_mlp_gradients", load().anova_mlp_gradients(self.handle, ctypes.c_void_p(X.data_ptr()),
                                                                 ctypes.c_void_p(y.data_ptr()), int(X.shape[0]),
                                                                 float(pos_weight), ctypes.byref(loss)))
        return loss.value

    def train(self, X, y, batch: int = 4096, epochs: int = 10, lr: float = 1e-3, pos_weight: float = 1.0):
        import numpy as np
        hist = np.zeros(epochs)
        _check("anova_mlp_train", load().anova_mlp_train(self.handle, ctypes.c_void_p(X.data_ptr()),
                                                         ctypes.c_void_p(y.data_ptr()), int(X.shape[0]), int(batch),
                                                         int(epochs), float(lr), float(pos_weight),
                                                         ctypes.c_void_p(hist.ctypes.data)))
        return hist


def mlp_init_params(seed: int, n_features: int = N_SCREEN_FEATURES, hidden: int = 128):
    """He-normal weights, zero biases, packed W1 | b1 | W2 | b2 | W3 | b3."""
    import numpy as np
    from . import inputs
    F, H = n_features, hidden
    w1 = inputs.normal(seed, 71, F * H) * np.sqrt(2.0 / F)
    w2 = inputs.normal(seed, 72, H * H) * np.sqrt(2.0 / H)
    w3 = inputs.normal(seed, 73, H) * np.sqrt(1.0 / H)
    return np.concatenate([w1, np.zeros(H), w2, np.zeros(H), w3, np.zeros(1)]).astype(np.float32)


def screen_features(plan: "Plan", y, fhat, lam: float, lam_prev: float, w=None):
    import torch
    X = torch.empty((len(plan.terms), N_SCREEN_FEATURES), dtype=torch.float32, device=plan.device)
    _check("anova_screen_features", load().anova_screen_features(
        plan.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(plan._weights(w) or None),
        ctypes.c_void_p(fhat.data_ptr()), float(lam), float(lam_prev), ctypes.c_void_p(X.data_ptr())))
    return X


def fista_screened_path(plan: "Plan", mlp: Mlp, y, lambdas, max_it=500, tol=1e-6, threshold=0.5, kkt_tol=1e-3,
                        w=None):
    """Screened group-lasso path; returns (path [n_lambda, n_coeffs], infos, stats)."""
    import torch
    n = len(lambdas)
    path = torch.zeros((n, plan.n_coeffs), dtype=plan.cplx, device=plan.device)
    lam = (ctypes.c_double * n)(*[float(v) for v in lambdas])
    infos = (SolveInfo * n)()
    st = ScreenStats()
    _check("fista_screened_path", load().fista_screened_path(
        plan.handle, mlp.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(plan._weights(w) or None), lam, n,
        int(max_it), float(tol), float(threshold), float(kkt_tol), ctypes.c_void_p(path.data_ptr()), infos,
        ctypes.byref(st)))
    return path, [infos[i].as_dict() for i in range(n)], st.as_dict()


def screening_training_set(plan: "Plan", y, lambdas, path, w=None):
    """Features and labels along a solved path (labels: group nonzero at the next lambda)."""
    import torch
    lam = sorted([float(v) for v in lambdas], reverse=True)
    order = sorted(range(len(lambdas)), key=lambda i: -float(lambdas[i]))
    Xs, ys = [], []
    prev = torch.zeros(plan.n_coeffs, dtype=plan.cplx, device=plan.device)
    lam_prev = lam[0]
    for j, i in enumerate(order):
        Xs.append(screen_features(plan, y, prev, lam[j], lam_prev, w))
        lab = torch.zeros(len(plan.terms), dtype=torch.float32, device=plan.device)
        for u in range(len(plan.terms)):
            o, ln = plan.term_offset(u)
            lab[u] = float(bool(torch.any(path[i, o:o + ln] != 0)))
        ys.append(lab)
        prev = path[i].contiguous()
        lam_prev = lam[j]
    return torch.cat(Xs).contiguous(), torch.cat(ys).contiguous()


# --------------------------------------------------------------- batches --

class Batch:
    """Independent problems run by one launch per kernel; vectors concatenated."""

    def __init__(self, xs, terms_list, bandwidths_list, stream=None):
        import torch
        P = len(xs)
        self.P = P
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._xs = [x.to(torch.float32).contiguous() for x in xs]
        self.terms = [[tuple(u) for u in t] for t in terms_list]
        d = (ctypes.c_int * P)(*[int(x.shape[0]) for x in self._xs])
        M = (ctypes.c_int64 * P)(*[int(x.shape[1]) for x in self._xs])
        xp = (ctypes.c_void_p * P)(*[x.data_ptr() for x in self._xs])
        nt = (ctypes.c_int * P)(*[len(t) for t in self.terms])
        self._td, self._bw = [], []
        for t, b in zip(self.terms, bandwidths_list):
            td = (ctypes.c_int32 * (3 * len(t)))()
            bw = (ctypes.c_int32 * len(t))()
            for i, u in enumerate(t):
                for j in range(3):
                    td[3 * i + j] = u[j] if j < len(u) else -1
                bw[i] = int(b[i]) if len(u) else 0
            self._td.append(td)
            self._bw.append(bw)
        i32p = ctypes.POINTER(ctypes.c_int32)
        tdp = (i32p * P)(*[ctypes.cast(t, i32p) for t in self._td])
        bwp = (i32p * P)(*[ctypes.cast(b, i32p) for b in self._bw])
        h = ctypes.c_void_p()
        _check("anova_batch_create", load().anova_batch_create(ctypes.byref(h), P, d, M, xp, nt, tdp, bwp, None,
                                                               ctypes.c_void_p(self.stream.cuda_stream or None)))
        self.handle = h
        no = (ctypes.c_int64 * (P + 1))()
        co = (ctypes.c_int64 * (P + 1))()
        _check("anova_batch_layout", load().anova_batch_layout(h, no, co))
        self.node_off = [no[i] for i in range(P + 1)]
        self.coef_off = [co[i] for i in range(P + 1)]
        self.device = self._xs[0].device

    def close(self):
        if getattr(self, "handle", None):
            load().anova_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def trafo(self, fhat):
        import torch
        out = torch.empty(self.node_off[-1], dtype=torch.complex64, device=self.device)
        _check("grouped_trafo_batch", load().grouped_trafo_batch(self.handle, ctypes.c_void_p(fhat.data_ptr()),
                                                                 ctypes.c_void_p(out.data_ptr())))
        return out

    def adjoint(self, y):
        import torch
        out = torch.empty(self.coef_off[-1], dtype=torch.complex64, device=self.device)
        _check("grouped_adjoint_batch", load().grouped_adjoint_batch(self.handle, ctypes.c_void_p(y.data_ptr()),
                                                                     ctypes.c_void_p(out.data_ptr())))
        return out

    def lsqr(self, y, lam, max_it=30):
        import torch
        out = torch.empty(self.coef_off[-1], dtype=torch.complex64, device=self.device)
        infos = (SolveInfo * self.P)()
        rc = load().lsqr_solve_batch(self.handle, ctypes.c_void_p(y.data_ptr()), float(lam), int(max_it),
                                     ctypes.c_void_p(out.data_ptr()), infos)
        if rc not in (0, -5):
            _check("lsqr_solve_batch", rc)
        return out, [infos[i].as_dict() for i in range(self.P)], rc

