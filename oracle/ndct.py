"""Direct FP64 sums of the grouped cosine transform (oracle; test infrastructure only).

The half-period cosine system of Sec. 5 on the cube [0, 1]^d,

    phi_k(x) = sqrt(2)^{|supp k|} prod_{j in supp k} cos(pi k_j x_j),   k in N_0^d,

grouped as in the Remark on other orthonormal systems (Sec. 3) and eq.
(appl:bandwidths): the block of a term u holds the k with supp k = u and
1 <= k_j <= N_u - 1, i.e. (N_u - 1)^{|u|} coefficients.  Block order follows
the term order; inside a block the multi-index over the term's sorted
coordinates is row-major (last fastest), each coordinate running 1..N_u - 1.
The empty term is the single k = 0 coefficient (phi_0 = 1).

    forward   f_j = sum_u sum_{k in block u} fhat_k phi_k(x_j)
    adjoint   g_k = sum_j y_j phi_k(x_j)          (phi_k is real: no conjugate)

computed straight from the definition with one table cos(pi k x_t) per node
and coordinate and a product over the term's coordinates (numpy einsum).
Nothing here is shared with the CUDA path.
"""
from __future__ import annotations

import string

import numpy as np


def block_sizes(terms, bandwidths) -> list[int]:
    return [1 if len(u) == 0 else (int(N) - 1) ** len(u) for u, N in zip(terms, bandwidths)]


def n_coeffs(terms, bandwidths) -> int:
    return int(sum(block_sizes(terms, bandwidths)))


def _table(xt: np.ndarray, N: int) -> np.ndarray:
    """sqrt(2) cos(pi k x_t) for k = 1..N-1: [M][N-1]."""
    k = np.arange(1, N, dtype=np.float64)
    return np.sqrt(2.0) * np.cos(np.pi * np.outer(np.asarray(xt, dtype=np.float64), k))


def trafo(x, terms, bandwidths, fhat) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    fhat = np.asarray(fhat, dtype=np.complex128)
    M = x.shape[1]
    f = np.zeros(M, dtype=np.complex128)
    off = 0
    for u, N, ln in zip(terms, bandwidths, block_sizes(terms, bandwidths)):
        blk = fhat[off:off + ln]
        off += ln
        s = len(u)
        if s == 0:
            f += blk[0]
            continue
        tabs = [_table(x[t], N) for t in u]
        idx = string.ascii_lowercase[:s]
        expr = ",".join("z" + c for c in idx) + "," + idx + "->z"
        f += np.einsum(expr, *tabs, blk.reshape((N - 1,) * s))
    return f


def adjoint(x, terms, bandwidths, y) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.complex128)
    out = []
    for u, N in zip(terms, bandwidths):
        s = len(u)
        if s == 0:
            out.append(np.array([np.sum(y)]))
            continue
        tabs = [_table(x[t], N) for t in u]
        idx = string.ascii_lowercase[:s]
        expr = "z," + ",".join("z" + c for c in idx) + "->" + idx
        out.append(np.einsum(expr, y, *tabs).reshape(-1))
    return np.concatenate(out)


def matrix(x, terms, bandwidths) -> np.ndarray:
    """The dense matrix [phi_k(x_j)]_{j,k} (columns in the block layout)."""
    x = np.asarray(x, dtype=np.float64)
    cols = []
    for u, N in zip(terms, bandwidths):
        s = len(u)
        if s == 0:
            cols.append(np.ones((x.shape[1], 1)))
            continue
        tabs = [_table(x[t], N) for t in u]
        prod = tabs[0]
        for tb in tabs[1:]:
            prod = (prod[:, :, None] * tb[:, None, :]).reshape(x.shape[1], -1)
        cols.append(prod)
    return np.concatenate(cols, axis=1).astype(np.complex128)
