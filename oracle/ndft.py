"""Direct FP64 summation of F and F^H (oracle; test infrastructure only).

Thin ctypes wrapper around ``ndft.c``; see that file for the definition it
implements (Definition "grouped Fourier transform" and eq. (FM), Sec. 3, and
the stacked adjoint of Sec. 3).  The shared object is compiled with gcc on
first use (or by ``build()``) next to the source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import anova

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ndft.c")
_LIB = os.path.join(_HERE, "_ndft.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ndft.c into _ndft.so (plain C, -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load(path: str | None = None):
    """Load the compiled summation library (``path`` overrides, used by mutation tests)."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    lib = ctypes.CDLL(path or build())
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
    common = [ctypes.c_int, ctypes.c_int64, f64p, ctypes.c_int, i32p, i32p, i32p, i64p]
    lib.oracle_grouped_trafo.argtypes = common + [f64p, f64p, ctypes.c_int]
    lib.oracle_grouped_adjoint.argtypes = common + [f64p, f64p, ctypes.c_int]
    lib.oracle_fourier_matrix.argtypes = common + [ctypes.c_int64, f64p, ctypes.c_int]
    for fn in (lib.oracle_grouped_trafo, lib.oracle_grouped_adjoint, lib.oracle_fourier_matrix):
        fn.restype = ctypes.c_int
    lib.oracle_max_order.restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def _prep(x, terms, bandwidths, lib):
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim != 2:
        raise ValueError("nodes must be [d][M]")
    order, dims, N = anova.term_arrays(terms, bandwidths, lib.oracle_max_order())
    offs, _ = anova.layout(terms, bandwidths)
    return x, order, dims, N, np.ascontiguousarray(offs)


def _as_interleaved(z, n):
    z = np.asarray(z, dtype=np.complex128).reshape(-1)
    if z.size != n:
        raise ValueError("vector length mismatch")
    return np.ascontiguousarray(z).view(np.float64)


def trafo(x, terms, bandwidths, fhat, threads: int | None = None, lib=None) -> np.ndarray:
    """f = F(X, I_N(U)) fhat by direct summation (Definition, Sec. 3)."""
    lib = lib or load()
    x, order, dims, N, offs = _prep(x, terms, bandwidths, lib)
    d, M = x.shape
    c = _as_interleaved(fhat, anova.n_coeffs(terms, bandwidths))
    out = np.zeros(2 * M)
    rc = lib.oracle_grouped_trafo(d, M, x, len(terms), order, dims, N, offs, c, out,
                                  threads or default_threads())
    if rc:
        raise ValueError(f"oracle_grouped_trafo: bad arguments ({rc})")
    return out.view(np.complex128)


def adjoint(x, terms, bandwidths, y, threads: int | None = None, lib=None) -> np.ndarray:
    """fhat = F(X, I_N(U))^H y by direct summation (stacked adjoint, Sec. 3)."""
    lib = lib or load()
    x, order, dims, N, offs = _prep(x, terms, bandwidths, lib)
    d, M = x.shape
    yy = _as_interleaved(y, M)
    out = np.zeros(2 * anova.n_coeffs(terms, bandwidths))
    rc = lib.oracle_grouped_adjoint(d, M, x, len(terms), order, dims, N, offs, yy, out,
                                    threads or default_threads())
    if rc:
        raise ValueError(f"oracle_grouped_adjoint: bad arguments ({rc})")
    return out.view(np.complex128)


def matrix(x, terms, bandwidths, threads: int | None = None, lib=None) -> np.ndarray:
    """The dense Fourier matrix F(X, I_N(U)) of eq. (FM), columns in layout order."""
    lib = lib or load()
    x, order, dims, N, offs = _prep(x, terms, bandwidths, lib)
    d, M = x.shape
    n = anova.n_coeffs(terms, bandwidths)
    out = np.zeros(2 * M * n)
    rc = lib.oracle_fourier_matrix(d, M, x, len(terms), order, dims, N, offs, n, out,
                                   threads or default_threads())
    if rc:
        raise ValueError(f"oracle_fourier_matrix: bad arguments ({rc})")
    return out.view(np.complex128).reshape(M, n)
