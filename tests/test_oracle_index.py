"""Pins of the oracle's index-set bookkeeping against numbers printed in the paper."""
import json
import os

import numpy as np
import pytest

from oracle import anova

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cardinalities.json")))


def _bw(terms, by_order):
    return [0 if len(u) == 0 else by_order[str(len(u))] for u in terms]


@pytest.mark.parametrize("case", GOLD["cases"], ids=lambda c: c["cite"][:24])
def test_paper_cardinalities(case):
    terms = anova.term_set(case["d"], case["ds"])
    assert len(terms) == case["n_terms"]
    assert anova.n_coeffs(terms, _bw(terms, case["N_by_order"])) == case["n_coeffs"]


@pytest.mark.parametrize("name", [k for k in GOLD["configs"] if not k.startswith("_")])
def test_config_counts(name):
    c = GOLD["configs"][name]
    terms = anova.term_set(c["d"], c["ds"])
    assert len(terms) == c["n_terms"]
    assert anova.n_coeffs(terms, _bw(terms, c["N_by_order"])) == c["n_coeffs"]


def test_term_order_and_downward_closed():
    terms = anova.term_set(5, 3)
    assert terms[0] == ()
    assert terms[1:6] == [(0,), (1,), (2,), (3,), (4,)]
    assert terms[6] == (0, 1) and terms[15] == (3, 4) and terms[16] == (0, 1, 2)
    s = set(terms)
    for u in terms:  # every subset of a term is a term (subset of ANOVA terms, Sec. 2)
        for r in range(len(u)):
            import itertools
            for v in itertools.combinations(u, r):
                assert v in s
    orders = [len(u) for u in terms]
    assert orders == sorted(orders)


def test_one_dim_set_is_asymmetric():
    # I_N = Z cap [-N/2, N/2): contains -N/2, not N/2 (Sec. 2)
    k = anova.one_dim_nonzero(8)
    assert list(k) == [-4, -3, -2, -1, 1, 2, 3]
    assert list(anova.one_dim_nonzero(2)) == [-1]
    with pytest.raises(ValueError):
        anova.one_dim_nonzero(7)


def test_frequencies_supports_and_distinct():
    d = 5
    terms = anova.term_set(d, 3)
    bw = [0] + [6] * 5 + [4] * 10 + [4] * 10
    K = anova.frequencies(terms, bw, d)
    assert K.shape == (anova.n_coeffs(terms, bw), d)
    offs, lens = anova.layout(terms, bw)
    for u, o, n, N in zip(terms, offs, lens, bw):
        blk = K[o:o + n]
        supp = blk != 0
        assert np.all(supp[:, list(u)]) and not np.any(np.delete(supp, list(u), axis=1))
        if len(u):
            assert blk[:, list(u)].min() >= -N // 2 and blk[:, list(u)].max() <= N // 2 - 1
    assert len({tuple(r) for r in K}) == K.shape[0]
    # row-major, last coordinate fastest
    o = offs[6]  # term (0, 1) with N = 4: values -2, -1, 1
    assert [tuple(K[o + i, :2]) for i in range(4)] == [(-2, -2), (-2, -1), (-2, 1), (-1, -2)]
