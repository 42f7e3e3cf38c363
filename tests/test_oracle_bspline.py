"""Pins of the paper's test function (Sec. 4, eq. (testfun)) as the input
generator produces it, and of the oracle's error measure (eq. (L2error)) and
Sobol indices (eq. (gsi)) on it.

What fixes the values here is the paper's text, not the code under test:
* the constants c_2, c_4, c_6 make ||B_j|| = 1 (stated after eq. (testfun));
* the Fourier coefficients of B_j are c_j sinc^j(pi k / j) cos(pi k)
  (checked by quadrature of the directly evaluated spline);
* the ANOVA terms of eq. (onedimterm), (twodimterm), (threedimterm) and the
  constant term sum to f, and vanish outside P({1,3,8}) u P({2,5,6}) u P({4,7,9});
* the variances of those terms give the Sobol indices in closed form;
* Parseval's identity of eq. (L2error) against a tensor-grid quadrature that
  is exact for trigonometric polynomials.
"""
import math

import numpy as np
import pytest

from oracle import anova, ndft, solvers
from paper_2010_10199_gb300 import inputs

C = inputs.BSPLINE_C
P3 = C[2] * C[4] * C[6]


def _gauss_legendre_pieces(j, n_nodes=16):
    """Nodes and weights on [0, 1) split at the spline's knots l / j."""
    t, w = np.polynomial.legendre.leggauss(n_nodes)
    xs, ws = [], []
    for l in range(j):
        a, b = l / j, (l + 1) / j
        xs.append(0.5 * (b - a) * t + 0.5 * (a + b))
        ws.append(0.5 * (b - a) * w)
    return np.concatenate(xs), np.concatenate(ws)


@pytest.mark.parametrize("j", [2, 4, 6])
def test_spline_norm_is_one(j):
    # B_j^2 is a polynomial of degree 2j - 2 <= 10 on each piece: 16-point rule is exact
    x, w = _gauss_legendre_pieces(j)
    assert abs(np.sum(w * inputs.bspline_B(j, x) ** 2) - 1.0) < 1e-13


@pytest.mark.parametrize("j", [2, 4, 6])
def test_spline_fourier_coefficients_match_the_paper(j):
    x, w = _gauss_legendre_pieces(j, 48)
    b = inputs.bspline_B(j, x)
    for k in range(-12, 13):
        ck = np.sum(w * b * np.exp(-2j * np.pi * k * x))
        a = np.pi * k / j
        paper = C[j] * (1.0 if k == 0 else (math.sin(a) / a) ** j) * math.cos(np.pi * k)
        assert abs(ck - paper) < 1e-12, (j, k)


def _anova_terms_paper(x):
    """The constant, one-, two- and three-dimensional ANOVA terms written out
    from eq. (onedimterm), (twodimterm), (threedimterm) (0-based coordinates):
    returns a dict term -> values at the nodes."""
    o = inputs.BSPLINE_ORDER
    g = {i: inputs.bspline_B(o[i], x[i]) - C[o[i]] for i in range(9)}
    out = {(): np.full(x.shape[1], 3.0 * P3)}
    for t in inputs.BSPLINE_TRIPLES:
        for i in t:
            out[(i,)] = P3 / C[o[i]] * g[i]
        for a in range(3):
            for b in range(a + 1, 3):
                i, k = sorted((t[a], t[b]))
                out[(i, k)] = P3 / (C[o[i]] * C[o[k]]) * g[i] * g[k]
        out[tuple(sorted(t))] = g[t[0]] * g[t[1]] * g[t[2]]
    return out


def test_anova_terms_sum_to_the_function():
    x = inputs.uniform_points(41, 9, 3000)
    terms = _anova_terms_paper(x)
    assert len(terms) == 1 + 9 + 9 + 3   # the active set U* of the paper
    assert np.max(np.abs(sum(terms.values()) - inputs.bspline_function(x))) < 1e-12


def test_coefficients_vanish_outside_the_active_set():
    terms = inputs.terms_up_to(9, 3)
    bw = inputs.bandwidths_by_order(terms, inputs.BSPLINE_SMALL_N)
    c = inputs.bspline_coefficients(terms, bw)
    offs, lens = anova.layout(terms, bw)
    active = set(_anova_terms_paper(np.zeros((9, 1))).keys())
    for u, o, n in zip(terms, offs, lens):
        nz = np.any(c[o:o + n] != 0)
        assert nz == (tuple(u) in active), u


def test_partial_sum_with_exact_coefficients_approximates_f():
    """sum_{k in I} c_k e^{2 pi i k x} with the generator's coefficient vector
    (its block layout included) against f at random nodes: the mean squared
    difference equals the Parseval tail ||f||^2 - sum_I |c_k|^2 up to the Monte
    Carlo error; a wrong sign, shift or layout breaks it by orders of magnitude."""
    terms = inputs.terms_up_to(9, 3)
    bw = inputs.bandwidths_by_order(terms, {1: 128, 2: 32, 3: 16})
    c = inputs.bspline_coefficients(terms, bw)
    x = inputs.uniform_points(42, 9, 20000)
    s = ndft.trafo(x, terms, bw, c)
    mse = float(np.mean(np.abs(inputs.bspline_function(x) - s) ** 2))
    tail = inputs.bspline_norm2() - float(np.sum(np.abs(c) ** 2))
    assert tail > 0
    assert 0.7 * tail < mse < 1.4 * tail, (mse, tail)
    assert tail / inputs.bspline_norm2() < 2e-4


def test_sobol_indices_of_the_exact_coefficients():
    """rho(u) from eq. (gsi): sigma^2(f_u) from the terms of eq. (onedimterm)
    etc. (e.g. (P / c_o(i))^2 (1 - c_o(i)^2) for u = {i}, since ||B_j|| = 1 and
    its mean is c_j), sigma^2(f) = 3 (1 - P^2).  The oracle's indices of the
    truncated exact coefficients approach them as the bandwidths grow."""
    o = inputs.BSPLINE_ORDER
    var_f = 3.0 * (1.0 - P3 ** 2)

    def exact(u):
        if len(u) == 0:
            return 0.0
        t = next((t for t in inputs.BSPLINE_TRIPLES if set(u) <= set(t)), None)
        if t is None:
            return 0.0
        v = 1.0
        for i in t:
            v *= (1.0 - C[o[i]] ** 2) if i in u else C[o[i]] ** 2
        return v / var_f

    terms = inputs.terms_up_to(9, 3)
    bw = inputs.bandwidths_by_order(terms, {1: 512, 2: 64, 3: 24})
    c = inputs.bspline_coefficients(terms, bw)
    offs, lens = anova.layout(terms, bw)
    rho = solvers.sobol_indices(c, offs, lens)
    ex = np.array([exact(u) for u in terms])
    assert abs(sum(ex) - 1.0) < 1e-12
    assert np.max(np.abs(rho - ex)) < 2e-3
    assert solvers.active_set(rho, terms, [1e-4, 1e-4, 1e-4]) == [i for i, e in enumerate(ex) if e > 0 or i == 0]


def test_l2_error_matches_tensor_grid_quadrature():
    """eq. (L2error) through Parseval against the mean of |f - S f|^2 over an
    L^3 tensor grid, exact for trigonometric polynomials of degree < L: a
    random 'function' with coefficients on a large index set, approximated on
    a smaller one."""
    d = 3
    terms = inputs.terms_up_to(d, 3)
    big = inputs.bandwidths_by_order(terms, {1: 10, 2: 8, 3: 6})
    small = inputs.bandwidths_by_order(terms, {1: 6, 2: 4, 3: 4})
    cf = inputs.complex_normal(3, 2, anova.n_coeffs(terms, big))
    fhat = inputs.complex_normal(4, 2, anova.n_coeffs(terms, small))
    # the exact coefficients restricted to the small set (frequency by frequency)
    kb = anova.frequencies(terms, big, d)
    ks = anova.frequencies(terms, small, d)
    lookup = {tuple(k): i for i, k in enumerate(kb)}
    c_small = np.array([cf[lookup[tuple(k)]] for k in ks])
    L = 12
    g = (np.arange(L) / L) - 0.5
    X = np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1)
    diff = ndft.trafo(X, terms, big, cf) - ndft.trafo(X, terms, small, fhat)
    quad = math.sqrt(float(np.mean(np.abs(diff) ** 2)) / float(np.sum(np.abs(cf) ** 2)))
    par = solvers.l2_error(fhat, c_small, float(np.sum(np.abs(cf) ** 2)))
    assert abs(par - quad) < 1e-12 * max(1.0, quad)


def test_l2_error_pins_catch_planted_mistakes():
    c = np.array([1.0, 2.0, -1.0j])
    fh = np.array([1.5, 2.0, 0.0])
    norm2 = 7.0   # ||f||^2 > sum |c|^2 = 6
    good = solvers.l2_error(fh, c, norm2)
    assert abs(good - math.sqrt((7.0 + 0.25 + 1.0 - 6.0) / 7.0)) < 1e-15
    bad_sign = math.sqrt(abs(7.0 - 1.25 + 6.0) / 7.0)                   # the two sums swapped in sign
    bad_unsquared = math.sqrt((7.0 + 0.5 + 1.0 - 6.0) / 7.0)            # |fhat - c| without the square
    assert abs(good - bad_sign) > 1e-3 and abs(good - bad_unsquared) > 1e-3
