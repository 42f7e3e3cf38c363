"""Index-set bookkeeping of the grouped transform (oracle; test infrastructure only).

* U_{d_s} = {u subset D : |u| <= d_s}                         -- Sec. 2, eq. (pizmosch)
* I_N = Z cap [-N/2, N/2), N even                              -- Sec. 2, before eq. (metallica)
* I_N^{u,d} = {k : supp k = u, k_j in I_N}, |I_N^{u,d}| = (N-1)^|u|
                                                               -- eq. (metallica), Remark (cardinality)
* I_N(U) = disjoint union over u in U                          -- eq. (groupedset)
* block order of F = [F_{u_1} F_{u_2} ...]                     -- eq. (bananarama)

The paper leaves the order of terms and coefficients open ("when introducing an
order on the sets u", after eq. (bananarama)).  The reading used here: the empty
set first, then by |u|, then lexicographically; inside a block, row-major over
the sorted coordinates of u with the last coordinate fastest, each coordinate
running -N/2..-1, 1..N/2-1.
"""
from __future__ import annotations

import itertools

import numpy as np


def term_set(d: int, ds: int) -> list[tuple[int, ...]]:
    """U_{d_s} over coordinates 0..d-1 in the order described above (eq. (pizmosch))."""
    out = [()]
    for s in range(1, ds + 1):
        out += list(itertools.combinations(range(d), s))
    return out


def one_dim_nonzero(N: int) -> np.ndarray:
    """I_N minus {0}: -N/2, ..., -1, 1, ..., N/2 - 1 (Remark (cardinality))."""
    if N % 2 or N < 2:
        raise ValueError("bandwidth must be even and >= 2 (N in 2N)")
    return np.array([k for k in range(-N // 2, N // 2) if k != 0], dtype=np.int64)


def group_size(u, N: int) -> int:
    """|I_N^{u,d}| = (N-1)^{|u|}; the empty set holds only k = 0."""
    return 1 if len(u) == 0 else (N - 1) ** len(u)


def layout(terms, bandwidths) -> tuple[np.ndarray, np.ndarray]:
    """Offsets and lengths of the coefficient blocks (eq. (groupedset), (bananarama))."""
    lens = np.array([group_size(u, N) for u, N in zip(terms, bandwidths)], dtype=np.int64)
    offs = np.zeros(len(lens), dtype=np.int64)
    if len(lens):
        offs[1:] = np.cumsum(lens)[:-1]
    return offs, lens


def n_coeffs(terms, bandwidths) -> int:
    return int(sum(group_size(u, N) for u, N in zip(terms, bandwidths)))


def frequencies(terms, bandwidths, d: int) -> np.ndarray:
    """All k in I_N(U) as rows of a [|I|, d] integer array, in layout order."""
    rows = []
    for u, N in zip(terms, bandwidths):
        if len(u) == 0:
            rows.append(np.zeros((1, d), dtype=np.int64))
            continue
        k1 = one_dim_nonzero(N)
        block = np.zeros(((N - 1) ** len(u), d), dtype=np.int64)
        for q, ell in enumerate(itertools.product(k1, repeat=len(u))):
            block[q, list(u)] = ell
        rows.append(block)
    return np.concatenate(rows, axis=0) if rows else np.zeros((0, d), dtype=np.int64)


def group_index(terms, bandwidths) -> np.ndarray:
    """Term id of every coefficient."""
    return np.concatenate([np.full(group_size(u, N), i, dtype=np.int64)
                           for i, (u, N) in enumerate(zip(terms, bandwidths))])


def term_arrays(terms, bandwidths, max_order: int):
    """Packed int32 arrays (order, dims[.., max_order], N) for the C summation."""
    n = len(terms)
    order = np.array([len(u) for u in terms], dtype=np.int32)
    dims = np.full((n, max_order), -1, dtype=np.int32)
    for i, u in enumerate(terms):
        if len(u) > max_order:
            raise ValueError("term order above the oracle's maximum")
        dims[i, :len(u)] = u
    N = np.array([max(int(b), 2) if len(u) else 2 for u, b in zip(terms, bandwidths)], dtype=np.int32)
    return order, dims, N
