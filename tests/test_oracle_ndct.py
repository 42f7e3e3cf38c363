"""Pins of the cosine oracle (oracle/ndct.py) against what the mathematics fixes.

* Orthonormality: on the L^d midpoint grid x_l = (l + 1/2) / L the functions
  phi_k of Sec. 5 with 1 <= k_j < L are orthonormal under (1/M) sum_j, so the
  matrix of a grouped cosine set satisfies Phi^T Phi = M I (different supports
  differ in a coordinate where one factor is 1 and the other sums to 0).
* One dimension reduces to the DCT-II: sum_l y_l cos(pi k (l + 1/2) / L) is
  half of scipy's unnormalised type-2 DCT.
* The exponential identity: prod_t cos(pi k_t x_t) = 2^{-s} sum over sign
  patterns eps of exp(2 pi i <eps k, x / 2>), so a cosine term equals the
  exponential oracle's term at the halved nodes with bandwidth 2N and the
  mirrored coefficients 2^{-s/2} fhat_{|k|}.
* Planted mistakes (normalisation dropped, 2 pi for pi, frequencies shifted by
  one) each fail the orthonormality pin.
"""
import numpy as np
import pytest

from oracle import ndct, ndft
from paper_2010_10199_gb300 import inputs


def _midpoint_grid(d, L):
    g = (np.arange(L) + 0.5) / L
    return np.array(np.meshgrid(*([g] * d), indexing="ij")).reshape(d, -1)


def _terms(d, ds, by_order):
    terms = inputs.terms_up_to(d, ds)
    return terms, inputs.bandwidths_by_order(terms, by_order) if ds else [0]


def test_orthonormal_on_midpoint_tensor_grid():
    d, L = 3, 9
    terms, bw = _terms(d, 3, {1: 9, 2: 7, 3: 5})
    X = _midpoint_grid(d, L)
    Phi = ndct.matrix(X, terms, bw)
    G = Phi.conj().T @ Phi
    assert Phi.shape == (L ** d, ndct.n_coeffs(terms, bw))
    assert np.max(np.abs(G - L ** d * np.eye(G.shape[0]))) < 1e-9


def test_matrix_forward_adjoint_agree():
    d = 4
    terms, bw = _terms(d, 3, {1: 12, 2: 6, 3: 4})
    x = inputs.uniform_points(5, d, 300) + 0.5          # nodes in [0, 1)^d
    f = inputs.complex_normal(6, 2, ndct.n_coeffs(terms, bw))
    y = inputs.complex_normal(7, 2, 300)
    Phi = ndct.matrix(x, terms, bw)
    assert np.max(np.abs(ndct.trafo(x, terms, bw, f) - Phi @ f)) < 1e-10
    assert np.max(np.abs(ndct.adjoint(x, terms, bw, y) - Phi.T @ y)) < 1e-10
    # adjointness with the real basis: <Phi f, y> = <f, Phi^T y> (bilinear form)
    assert abs(np.sum((Phi @ f) * y) - np.sum(f * ndct.adjoint(x, terms, bw, y))) < 1e-9


def test_one_dimension_is_the_dct_ii():
    scipy_fft = pytest.importorskip("scipy.fft")
    L, N = 40, 30
    x = ((np.arange(L) + 0.5) / L)[None, :]
    y = inputs.normal(8, 2, L)
    g = ndct.adjoint(x, [(0,)], [N], y)
    ref = np.sqrt(2.0) * scipy_fft.dct(y, type=2)[1:N] / 2.0
    assert np.max(np.abs(g - ref)) < 1e-12


def test_cosine_term_is_the_mirrored_exponential_term_at_half_nodes():
    d = 3
    x = inputs.uniform_points(9, d, 400) + 0.5
    for u, N in (((1,), 10), ((0, 2), 6), ((0, 1, 2), 5)):
        s = len(u)
        fh = inputs.complex_normal(10 + s, 2, (N - 1) ** s)
        # exponential coefficients on (I_{2N} minus 0)^s: -N..-1, 1..N-1 per coordinate
        k1 = [k for k in range(-N, N) if k != 0]
        g = np.zeros((2 * N - 1,) * s, dtype=np.complex128)
        blk = fh.reshape((N - 1,) * s)
        for idx in np.ndindex(*g.shape):
            ks = [k1[i] for i in idx]
            if all(k != 0 and abs(k) <= N - 1 for k in ks):
                g[idx] = 2.0 ** (-s / 2) * blk[tuple(abs(k) - 1 for k in ks)]
        cos_side = ndct.trafo(x, [u], [N], fh)
        exp_side = ndft.trafo(x / 2.0, [u], [2 * N], g.reshape(-1))
        assert np.max(np.abs(cos_side - exp_side)) < 1e-10, u


def test_orthonormality_pin_catches_planted_mistakes():
    d, L = 2, 8
    terms, bw = _terms(d, 2, {1: 8, 2: 5})
    X = _midpoint_grid(d, L)

    def gram_ok(tab):
        cols = []
        for u, N in zip(terms, bw):
            if len(u) == 0:
                cols.append(np.ones((X.shape[1], 1)))
                continue
            prod = tab(X[u[0]], N)
            for t in u[1:]:
                prod = (prod[:, :, None] * tab(X[t], N)[:, None, :]).reshape(X.shape[1], -1)
            cols.append(prod)
        Phi = np.concatenate(cols, axis=1)
        return np.max(np.abs(Phi.T @ Phi - L ** d * np.eye(Phi.shape[1]))) < 1e-9

    good = lambda xt, N: np.sqrt(2.0) * np.cos(np.pi * np.outer(xt, np.arange(1, N)))
    no_norm = lambda xt, N: np.cos(np.pi * np.outer(xt, np.arange(1, N)))
    two_pi = lambda xt, N: np.sqrt(2.0) * np.cos(2 * np.pi * np.outer(xt, np.arange(1, N)))
    shifted = lambda xt, N: np.sqrt(2.0) * np.cos(np.pi * np.outer(xt, np.arange(0, N - 1)))
    assert gram_ok(good)
    for bad in (no_norm, two_pi, shifted):
        assert not gram_ok(bad)
