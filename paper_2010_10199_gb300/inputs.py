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


# --------------------------------------------------------------------------
# the paper's test function (Sec. 4, eq. (testfun)), d = 9:
#   f(x) = B2(x1) B4(x3) B6(x8) + B2(x2) B4(x5) B6(x6) + B2(x4) B4(x7) B6(x9)
# with B_j(x) = c_j sum_k sinc^j(pi k / j) cos(pi k) exp(2 pi i k x).  That
# series is c_j times the periodised B-spline j M_j(j x) on [0, 1) (M_j the
# cardinal B-spline of order j on [0, j], whose Fourier transform is
# exp(-i w j / 2) sinc^j(w / 2)), which is how f is evaluated here.  This is
# data: the sampled values y and, for the error measure of eq. (L2error), the
# exact coefficients on a grouped index set.
# --------------------------------------------------------------------------

BSPLINE_C = {2: math.sqrt(3.0 / 4.0), 4: math.sqrt(315.0 / 604.0), 6: math.sqrt(277200.0 / 655177.0)}
# the three coordinate triples of the test function, 0-based ({1,3,8}, {2,5,6},
# {4,7,9} in the paper), each listed as (B2 coordinate, B4 coordinate, B6 coordinate)
BSPLINE_TRIPLES = ((0, 2, 7), (1, 4, 5), (3, 6, 8))
BSPLINE_ORDER = {c: j for t in BSPLINE_TRIPLES for c, j in zip(t, (2, 4, 6))}


def cardinal_bspline(j: int, t: np.ndarray) -> np.ndarray:
    """M_j(t) = 1/(j-1)! sum_{i=0}^{j} (-1)^i C(j, i) (t - i)_+^{j-1}, supported on [0, j]."""
    t = np.asarray(t, dtype=np.float64)
    s = np.zeros_like(t)
    for i in range(j + 1):
        s += (-1) ** i * math.comb(j, i) * np.maximum(t - i, 0.0) ** (j - 1)
    s /= math.factorial(j - 1)
    return np.where((t >= 0) & (t <= j), s, 0.0)


def bspline_B(j: int, x: np.ndarray) -> np.ndarray:
    """B_j of the test function at x on the torus (any real x)."""
    u = np.mod(np.asarray(x, dtype=np.float64), 1.0)
    return BSPLINE_C[j] * j * cardinal_bspline(j, j * u)


def bspline_function(x: np.ndarray) -> np.ndarray:
    """The test function of eq. (testfun) at nodes x [9][M]."""
    f = np.zeros(x.shape[1])
    for t in BSPLINE_TRIPLES:
        f += bspline_B(2, x[t[0]]) * bspline_B(4, x[t[1]]) * bspline_B(6, x[t[2]])
    return f


def bspline_coefficient_1d(j: int, k: np.ndarray) -> np.ndarray:
    """c_j sinc^j(pi k / j) cos(pi k): the k-th Fourier coefficient of B_j."""
    k = np.asarray(k, dtype=np.float64)
    a = np.pi * k / j
    sinc = np.where(k == 0, 1.0, np.sin(a) / np.where(k == 0, 1.0, a))
    return BSPLINE_C[j] * sinc ** j * np.cos(np.pi * k)


def bspline_coefficients(terms, bandwidths) -> np.ndarray:
    """Exact Fourier coefficients c_k(f) of the test function on I_N(U), in the
    block layout (term order; inside a block row-major over the term's sorted
    coordinates, last fastest, each coordinate -N/2..N/2-1 without 0).  A
    frequency with support u gets the sum over the triples T containing u of
    prod_{i in u} c_{o(i)}(k_i) prod_{i in T minus u} c_{o(i)}."""
    out = []
    for u, N in zip(terms, bandwidths):
        s = len(u)
        if s == 0:
            out.append(np.array([sum(BSPLINE_C[2] * BSPLINE_C[4] * BSPLINE_C[6] for _ in BSPLINE_TRIPLES)]))
            continue
        k1 = np.array([k for k in range(-N // 2, N // 2) if k != 0], dtype=np.float64)
        block = np.zeros((N - 1) ** s)
        for t in BSPLINE_TRIPLES:
            if not set(u) <= set(t):
                continue
            const = 1.0
            for c in t:
                if c not in u:
                    const *= BSPLINE_C[BSPLINE_ORDER[c]]
            grids = np.meshgrid(*[bspline_coefficient_1d(BSPLINE_ORDER[c], k1) for c in u], indexing="ij")
            prod = np.ones_like(grids[0])
            for g in grids:
                prod = prod * g
            block += const * prod.reshape(-1)
        out.append(block)
    return np.concatenate(out).astype(np.complex128)


def bspline_norm2() -> float:
    """||f||^2 = 3 + 6 (c_2 c_4 c_6)^2 (each triple has norm 1; two different
    triples share no coordinate, so their inner product is the product of
    their means)."""
    p = BSPLINE_C[2] * BSPLINE_C[4] * BSPLINE_C[6]
    return 3.0 + 6.0 * p * p


# bandwidths of the LSQR and FISTA experiments (i)/(ii) and (iii)/(iv):
# eq. (smallbandwidths) and eq. (largebandwidths)
BSPLINE_SMALL_N = {1: 26, 2: 6, 3: 4}
BSPLINE_LARGE_N = {1: 352, 2: 20, 3: 8}


def bspline_workload(seed: int = 0, M: int = 10_000, bandwidths=None, noise: float = 0.0) -> dict:
    """The experiments of Sec. 4: M i.i.d. uniform nodes on the torus (here
    [-1/2, 1/2)^9), y = f(x) + noise * sqrt(mean f(x)^2) * N(0, 1), all terms
    with |u| <= 3 and the small bandwidths of eq. (smallbandwidths) unless
    others are given; also the exact coefficients on I_N(U_3) and ||f||^2."""
    d = 9
    by_order = BSPLINE_SMALL_N if bandwidths is None else bandwidths
    terms = terms_up_to(d, 3)
    bw = bandwidths_by_order(terms, by_order)
    x = uniform_points(seed, d, M)
    fx = bspline_function(x)
    y = fx + noise * math.sqrt(float(np.mean(fx ** 2))) * normal(seed, S_NOISE, M)
    return dict(name="bspline", d=d, M=M, terms=terms, bandwidths=bw, x=x, y=y.astype(np.complex128),
                c=bspline_coefficients(terms, bw), norm2=bspline_norm2(), noise=noise)


# --------------------------------------------------------------------------
# the cosine (non-periodic) workload: the shape of the application of Sec. 5
# (d = 12 attributes min-max normalised into [0, 1], all terms with |u| <= 2,
# N = 82 / 10 as in eq. (appl:bandwidths): 79 terms, 6 319 coefficients,
# 36 160 training nodes, labels y in {0, 1}).  The census data are not here;
# synthetic attributes stand in: six continuous ones (Beta(2,5)-skewed and
# uniform) and six categorical ones with 2..16 levels spread over [0, 1], and
# a label that thresholds a sparse low-order function of them plus noise.
# --------------------------------------------------------------------------

def cosine_workload(seed: int = 0, M: int = 36_160, bandwidths=None) -> dict:
    d = 12
    by_order = {1: 82, 2: 10} if bandwidths is None else bandwidths
    terms = terms_up_to(d, 2)
    bw = bandwidths_by_order(terms, by_order)
    u = uniform(seed, S_POINTS, 3 * d * M).reshape(3, d, M)
    x = np.empty((d, M))
    for t in range(d):
        if t < 3:       # skewed continuous attribute: the median-of-3 order statistic of u^2
            x[t] = np.median(u[:, t, :] ** 2, axis=0)
        elif t < 6:     # uniform continuous attribute
            x[t] = u[0, t]
        else:           # categorical attribute with 2..16 levels, normalised to [0, 1]
            levels = 2 + (t * 5) % 15
            x[t] = np.floor(u[0, t] * levels) / (levels - 1)
    score = (np.sin(np.pi * x[0]) * x[7] + 0.8 * np.exp(-6 * (x[3] - 0.3) ** 2) + 0.5 * x[1] * x[9]
             + 0.3 * np.cos(2 * np.pi * x[4]) + 0.2 * normal(seed, S_NOISE, M))
    y = (score > np.median(score)).astype(np.float64)
    return dict(name="cosine_adult_shape", d=d, M=M, terms=terms, bandwidths=bw, x=x,
                y=y.astype(np.complex128))
