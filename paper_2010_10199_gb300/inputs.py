"""Seeded synthetic workloads for the grouped transform and its solvers.

This module generates inputs only: points, coefficient vectors, data vectors,
term lists and bandwidths.  It holds none of the method's arithmetic (no
Fourier sums, no windows, no solver steps), so both the CUDA path and the
FP64 oracle may consume what it produces without sharing any computation.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw ``i`` of stream ``(seed, stream)`` is
``mix(key(seed, stream) + (i + 1) * GAMMA)``.  Uniforms take the top 53 bits;
normals use the Box--Muller transform on pairs of uniforms.  Everything is
produced in FP64 on the host.

The workload shapes follow the paper's experiments (uniform i.i.d. nodes on the
torus, low-order ANOVA test functions with additive Gaussian noise, Sec. 4) at
the sizes of the five benchmark configurations:

* ``c1_small``   d=6,  |u|<=2, N=16/8,        M=2000
* ``c2_scale``   d=20, |u|<=2, N=64/32,       M=1e6
* ``c3_lsqr``    d=10, |u|<=3, N=100/24/10,   M=5e5, Beta(2,2) nodes
* ``c4_fista``   d=30, |u|<=2, N=32/16,       M=2e6
* ``c5_batched`` 64 problems, d in 5..15, |u|<=2, N=32/16, M log-uniform
"""
from __future__ import annotations

import itertools
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)

# stream ids (independent counter streams per quantity)
S_POINTS, S_COEFF, S_NOISE, S_Y, S_CHOICE, S_META = 1, 2, 3, 4, 5, 6


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


def splitmix64(state: int, n: int) -> np.ndarray:
    """First ``n`` outputs of the sequential SplitMix64 generator started at ``state``."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(state & 0xFFFFFFFFFFFFFFFF) + i * GAMMA)


def _key(seed: int, stream: int) -> int:
    return int(splitmix64((seed * 0x10001 + stream) & 0xFFFFFFFFFFFFFFFF, 1)[0])


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` doubles in [0, 1) from counter positions ``offset .. offset+n-1``."""
    key = np.uint64(_key(seed, stream))
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(key + i * GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """``n`` standard normals by Box--Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def complex_normal(seed: int, stream: int, n: int) -> np.ndarray:
    """(a + ib)/sqrt(2) with a, b i.i.d. N(0,1), so E|z|^2 = 1."""
    z = normal(seed, stream, 2 * n)
    return (z[0::2] + 1j * z[1::2]) / math.sqrt(2.0)


def uniform_points(seed: int, d: int, M: int, stream: int = S_POINTS) -> np.ndarray:
    """i.i.d. uniform nodes on [-1/2, 1/2)^d, FP64, SoA layout [d][M]."""
    return (uniform(seed, stream, d * M) - 0.5).reshape(d, M)


def beta22_points(seed: int, d: int, M: int, stream: int = S_POINTS) -> np.ndarray:
    """Beta(2,2) nodes shifted to [-1/2, 1/2): the median of three uniforms has
    exactly the Beta(2,2) law."""
    u = uniform(seed, stream, 3 * d * M).reshape(3, d * M)
    return (np.median(u, axis=0) - 0.5).reshape(d, M)


def choice(seed: int, stream: int, n: int, k: int, offset: int = 0) -> list[int]:
    """k distinct integers from range(n) (partial Fisher--Yates on the stream)."""
    u = uniform(seed, stream, k, offset)
    pool = list(range(n))
    out = []
    for i in range(k):
        j = i + int(u[i] * (n - i))
        pool[i], pool[j] = pool[j], pool[i]
        out.append(pool[i])
    return out


# --------------------------------------------------------------------------
# term lists and bandwidths (inputs of the plan; the layout rules themselves
# live separately in the oracle and in the CUDA plan)
# --------------------------------------------------------------------------

def terms_up_to(d: int, ds: int) -> list[tuple[int, ...]]:
    """All u subset of {0..d-1} with |u| <= ds: empty set first, then by |u|,
    then lexicographically (0-based coordinate ids)."""
    out: list[tuple[int, ...]] = [()]
    for s in range(1, ds + 1):
        out.extend(itertools.combinations(range(d), s))
    return out


def bandwidths_by_order(terms, by_order: dict[int, int]) -> list[int]:
    return [0 if len(u) == 0 else by_order[len(u)] for u in terms]


def gaussian_bump_sum(x: np.ndarray, groups: list[tuple[int, ...]]) -> np.ndarray:
    """sum over groups of prod_{t in group} exp(-8 x_t^2) (the test-function
    family of the benchmark configurations; 0-based coordinates)."""
    f = np.zeros(x.shape[1])
    for g in groups:
        p = np.ones(x.shape[1])
        for t in g:
            p *= np.exp(-8.0 * x[t] ** 2)
        f += p
    return f


def c1_function(x: np.ndarray) -> np.ndarray:
    """exp(-8 x1^2) exp(-8 x2^2) + sin(2 pi x3) + exp(-8 x4^2) cos(2 pi x5)
    (1-based coordinates as written in the configuration)."""
    return (np.exp(-8 * x[0] ** 2) * np.exp(-8 * x[1] ** 2)
            + np.sin(2 * np.pi * x[2])
            + np.exp(-8 * x[3] ** 2) * np.cos(2 * np.pi * x[4]))


def coeff_count(terms, bandwidths) -> int:
    """Number of unknowns, only needed to size random vectors here."""
    return sum(1 if len(u) == 0 else (N - 1) ** len(u) for u, N in zip(terms, bandwidths))


def decaying_coefficients(seed: int, terms, bandwidths) -> np.ndarray:
    """Complex coefficients N(0,1)/(1+|k|^2), |k|^2 = sum_t k_t^2 over the term's
    coordinates, in the block layout (term order, row-major over the term's
    sorted coordinates, last fastest, each coordinate -N/2..N/2-1 without 0)."""
    n = coeff_count(terms, bandwidths)
    z = complex_normal(seed, S_COEFF, n)
    scale = np.empty(n)
    pos = 0
    for u, N in zip(terms, bandwidths):
        s = len(u)
        if s == 0:
            scale[pos] = 1.0
            pos += 1
            continue
        k1 = np.array([k for k in range(-N // 2, N // 2) if k != 0], dtype=np.float64)
        grids = np.meshgrid(*([k1] * s), indexing="ij")
        k2 = sum(g ** 2 for g in grids).reshape(-1)
        scale[pos:pos + k2.size] = 1.0 / (1.0 + k2)
        pos += k2.size
    return z * scale


# --------------------------------------------------------------------------
# the five workload configurations
# --------------------------------------------------------------------------

def c1_small(seed: int = 0) -> dict:
    d, M = 6, 2000
    terms = terms_up_to(d, 2)
    bw = bandwidths_by_order(terms, {1: 16, 2: 8})
    x = uniform_points(seed, d, M)
    y = c1_function(x) + 0.01 * normal(seed, S_NOISE, M)
    return dict(name="c1_small", d=d, M=M, terms=terms, bandwidths=bw, x=x,
                y=y.astype(np.complex128), lam=1e-3, iters=50)


def c2_scale(seed: int = 0, M: int = 1_000_000) -> dict:
    d = 20
    terms = terms_up_to(d, 2)
    bw = bandwidths_by_order(terms, {1: 64, 2: 32})
    x = uniform_points(seed, d, M)
    fhat = decaying_coefficients(seed, terms, bw)
    y = complex_normal(seed, S_Y, M)
    return dict(name="c2_scale", d=d, M=M, terms=terms, bandwidths=bw, x=x,
                fhat=fhat, y=y)


def c3_lsqr(seed: int = 0, M: int = 500_000) -> dict:
    d = 10
    terms = terms_up_to(d, 3)
    bw = bandwidths_by_order(terms, {1: 100, 2: 24, 3: 10})
    x = beta22_points(seed, d, M)
    pairs = [tuple(sorted(choice(seed, S_CHOICE, d, 2, offset=8 * i))) for i in range(3)]
    triple = tuple(sorted(choice(seed, S_CHOICE, d, 3, offset=64)))
    y = gaussian_bump_sum(x, pairs + [triple]) + 0.01 * normal(seed, S_NOISE, M)
    lams = np.geomspace(1e0, 1e-4, 10)
    return dict(name="c3_lsqr", d=d, M=M, terms=terms, bandwidths=bw, x=x,
                y=y.astype(np.complex128), active=pairs + [triple], lambdas=lams)


def c4_fista(seed: int = 0, M: int = 2_000_000) -> dict:
    d = 30
    terms = terms_up_to(d, 2)
    bw = bandwidths_by_order(terms, {1: 32, 2: 16})
    x = uniform_points(seed, d, M)
    pairs = []
    i = 0
    while len(pairs) < 5:
        p = tuple(sorted(choice(seed, S_CHOICE, d, 2, offset=8 * i)))
        i += 1
        if p not in pairs:
            pairs.append(p)
    singles = [(c,) for c in choice(seed, S_CHOICE + 100, d, 3)]
    y = gaussian_bump_sum(x, pairs + singles) + 0.05 * normal(seed, S_NOISE, M)
    lams = np.geomspace(1e-1, 1e-5, 20)
    return dict(name="c4_fista", d=d, M=M, terms=terms, bandwidths=bw, x=x,
                y=y.astype(np.complex128), active=pairs + singles, lambdas=lams)


def c5_problem(p: int, scale: float = 1.0) -> dict:
    """Problem ``p`` of the many-problem batch (seed = p)."""
    u = uniform(p, S_META, 2)
    M = int(round(math.exp(math.log(1e4) + u[0] * (math.log(2e5) - math.log(1e4))) * scale))
    M = max(M, 1)
    d = 5 + int(u[1] * 11)
    terms = terms_up_to(d, 2)
    bw = bandwidths_by_order(terms, {1: 32, 2: 16})
    x = uniform_points(p, d, M)
    pair = tuple(sorted(choice(p, S_CHOICE, d, 2)))
    single = (choice(p, S_CHOICE + 100, d, 1)[0],)
    y = gaussian_bump_sum(x, [pair, single]) + 0.01 * normal(p, S_NOISE, M)
    return dict(name=f"c5_problem_{p}", d=d, M=M, terms=terms, bandwidths=bw, x=x,
                y=y.astype(np.complex128), lam=1e-3, iters=30)


def c5_batched(n_problems: int = 64, scale: float = 1.0) -> list[dict]:
    return [c5_problem(p, scale) for p in range(n_problems)]


def subsample(work: dict, m: int, seed: int = 12345) -> np.ndarray:
    """Sorted indices of an m-point subsample of a workload's nodes."""
    M = work["M"]
    if m >= M:
        return np.arange(M)
    u = uniform(seed, S_META + 7, m)
    idx = np.unique((u * M).astype(np.int64))
    return idx
