"""Pins of the FP64 direct summation (oracle) against facts that do not come from itself.

* one 1-D term on equispaced nodes is a length-N DFT: checked against numpy.fft
* on a full tensor grid with L >= N_u nodes per axis, F^H F = M I exactly
  (distinct frequencies differ in some coordinate by 0 < |dk| < L)
* adjointness <F f, y> = <f, F^H y>
* unit coefficient vectors reproduce exp(2 pi i <k, x>) evaluated with the full
  d-dimensional inner product (brute force on tiny inputs)
* block structure: F(X, I(U)) f = sum over terms of the single-term transforms
  (eq. (bananarama))
* mutation check: plausible mistakes planted in a copy of the C source are
  each caught by at least one of these pins
"""
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import anova, ndft
from paper_2010_10199_gb300 import inputs


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- pins ----

def pin_dft(lib):
    """f_j for x_j = j/N - 1/2 equals N * ifft of (fhat_k (-1)^k) placed at k mod N."""
    errs = []
    for N in (2, 8, 16, 64):
        x = (np.arange(N) / N - 0.5)[None, :]
        fh = inputs.complex_normal(N, 2, N - 1)
        f = ndft.trafo(x, [(0,)], [N], fh, lib=lib)
        a = np.zeros(N, dtype=np.complex128)
        k = anova.one_dim_nonzero(N)
        a[k % N] = fh * (-1.0) ** k
        ref = N * np.fft.ifft(a)
        errs.append(_rel(f, ref))
        # adjoint: fhat_k = sum_j y_j exp(-2 pi i k x_j) = (-1)^k * fft(y)[k mod N]
        y = inputs.complex_normal(N, 4, N)
        g = ndft.adjoint(x, [(0,)], [N], y, lib=lib)
        errs.append(_rel(g, np.fft.fft(y)[k % N] * (-1.0) ** k))
    return max(errs)


def pin_tensor_grid(lib):
    """F^H F = M I on an L^3 tensor grid, L = 8 >= every N_u, d = 3, all |u| <= 3."""
    d, L = 3, 8
    g = np.arange(L) / L - 0.5
    X = np.stack([a.reshape(-1) for a in np.meshgrid(g, g, g, indexing="ij")])
    terms = anova.term_set(d, 3)
    bw = [0, 8, 6, 8, 4, 6, 8, 4]
    F = ndft.matrix(X, terms, bw, lib=lib)
    G = F.conj().T @ F
    return np.abs(G - X.shape[1] * np.eye(G.shape[0])).max() / X.shape[1]


def pin_adjoint(lib):
    d, M = 4, 257
    x = inputs.uniform_points(3, d, M)
    terms = anova.term_set(d, 3)
    bw = [0] + [8] * 4 + [6] * 6 + [4] * 4
    n = anova.n_coeffs(terms, bw)
    fh = inputs.complex_normal(3, 2, n)
    y = inputs.complex_normal(3, 4, M)
    a = np.vdot(y, ndft.trafo(x, terms, bw, fh, lib=lib))
    b = np.vdot(ndft.adjoint(x, terms, bw, y, lib=lib), fh)
    return abs(a - b) / abs(a)


def pin_unit_vectors(lib):
    d, M = 4, 9
    x = inputs.uniform_points(5, d, M)
    terms = anova.term_set(d, 2)
    bw = [0] + [6] * 4 + [4] * 6
    K = anova.frequencies(terms, bw, d)
    n = K.shape[0]
    F = ndft.matrix(x, terms, bw, lib=lib)
    ref = np.exp(2j * np.pi * (x.T @ K.T))  # full inner products <k, x_j>
    err = np.abs(F - ref).max()
    # the transform of e_q is column q
    for q in (0, 1, n // 2, n - 1):
        e = np.zeros(n, dtype=np.complex128)
        e[q] = 1.0
        err = max(err, np.abs(ndft.trafo(x, terms, bw, e, lib=lib) - ref[:, q]).max())
    return err


def pin_blocks(lib):
    d, M = 5, 100
    x = inputs.uniform_points(8, d, M)
    terms = anova.term_set(d, 2)
    bw = [0] + [10] * 5 + [6] * 10
    offs, lens = anova.layout(terms, bw)
    fh = inputs.complex_normal(8, 2, anova.n_coeffs(terms, bw))
    total = ndft.trafo(x, terms, bw, fh, lib=lib)
    acc = np.zeros(M, dtype=np.complex128)
    for u, N, o, n in zip(terms, bw, offs, lens):
        acc += ndft.trafo(x, [u], [N], fh[o:o + n], lib=lib)
    return _rel(total, acc)


PINS = {"dft": (pin_dft, 1e-12), "tensor_grid": (pin_tensor_grid, 1e-12),
        "adjoint": (pin_adjoint, 1e-12), "unit_vectors": (pin_unit_vectors, 1e-12),
        "blocks": (pin_blocks, 1e-12)}


@pytest.mark.parametrize("name", list(PINS))
def test_pin(oracle_lib, name):
    fn, tol = PINS[name]
    assert fn(oracle_lib) < tol


def test_empty_term_only(oracle_lib):
    x = inputs.uniform_points(1, 3, 50)
    f = ndft.trafo(x, [()], [0], np.array([2.0 - 1.0j]), lib=oracle_lib)
    assert np.allclose(f, 2.0 - 1.0j, rtol=0, atol=0)
    y = inputs.complex_normal(1, 4, 50)
    g = ndft.adjoint(x, [()], [0], y, lib=oracle_lib)
    assert abs(g[0] - y.sum()) < 1e-13


def test_thread_count_invariance(oracle_lib):
    w = inputs.c1_small()
    fh = inputs.complex_normal(0, 2, anova.n_coeffs(w["terms"], w["bandwidths"]))
    a = ndft.trafo(w["x"], w["terms"], w["bandwidths"], fh, threads=1, lib=oracle_lib)
    b = ndft.trafo(w["x"], w["terms"], w["bandwidths"], fh, threads=5, lib=oracle_lib)
    assert np.array_equal(a, b)
    c = ndft.adjoint(w["x"], w["terms"], w["bandwidths"], w["y"], threads=1, lib=oracle_lib)
    e = ndft.adjoint(w["x"], w["terms"], w["bandwidths"], w["y"], threads=3, lib=oracle_lib)
    assert np.array_equal(c, e)


def test_rejects_bad_arguments(oracle_lib):
    x = inputs.uniform_points(1, 2, 4)
    with pytest.raises(ValueError):
        ndft.trafo(x, [(0,)], [7], np.zeros(6), lib=oracle_lib)
    with pytest.raises(ValueError):
        ndft.trafo(x, [(5,)], [4], np.zeros(3), lib=oracle_lib)


# ------------------------------------------------------------ mutations ----

MUTATIONS = {
    "sign_flip": (r"cos\(2\.0 \* M_PI \* r\);\n    \*s = sin\(2\.0 \* M_PI \* r\)",
                  "cos(2.0 * M_PI * r);\n    *s = -sin(2.0 * M_PI * r)"),
    "freq_keeps_zero": (r"return \(i < N / 2\) \? i - N / 2 : i - N / 2 \+ 1;",
                        "return i - N / 2;"),
    "adjoint_no_conj": (r"c\[2 \* q\] \+= yr \* er \+ yi \* ei;\n                c\[2 \* q \+ 1\] \+= yi \* er - yr \* ei;",
                        "c[2 * q] += yr * er - yi * ei;\n                c[2 * q + 1] += yi * er + yr * ei;"),
    "drop_empty_term": (r"ar \+= c\[0\];\n                    ai \+= c\[1\];",
                        "(void)c;"),
    "first_coordinate_only": (r"J->dims\[term \* MAX_ORDER \+ t\]", "J->dims[term * MAX_ORDER]"),
    "transposed_block": (r"\(size_t\)t \* 2 \* \(N - 1\) \+ 2 \* idx\[t\]",
                         "(size_t)t * 2 * (N - 1) + 2 * idx[s - 1 - t]"),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_pins_catch_planted_mistakes(tmp_path, name):
    src = open(os.path.join(os.path.dirname(ndft.__file__), "ndft.c")).read()
    pat, rep = MUTATIONS[name]
    mutated, n = re.subn(pat, rep, src)
    assert n >= 1, f"mutation {name} did not apply"
    c = tmp_path / "ndft_mut.c"
    c.write_text(mutated)
    so = tmp_path / "ndft_mut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
                           str(c), "-o", str(so), "-lm"])
    lib = ndft.load(str(so))
    caught = []
    for pname, (fn, tol) in PINS.items():
        try:
            caught.append(fn(lib) >= tol)
        except Exception:
            caught.append(True)
    # the empty-term pin is a separate test; use it for the dropped-term mutation
    if name == "drop_empty_term":
        x = inputs.uniform_points(1, 3, 5)
        f = ndft.trafo(x, [()], [0], np.array([1.0 + 0j]), lib=lib)
        caught.append(not np.allclose(f, 1.0))
    assert any(caught), f"no pin caught mutation {name}"
