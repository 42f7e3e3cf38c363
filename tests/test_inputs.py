"""The seeded input generators (no method arithmetic): published RNG values and laws."""
import numpy as np

from paper_2010_10199_gb300 import inputs


def test_splitmix64_published_first_output():
    # SplitMix64 seeded with 0: first output 0xE220A8397B1DCDAF (Steele, Lea, Flood 2014;
    # the value printed by the public splitmix64.c reference generator)
    assert int(inputs.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF


def test_uniform_and_normal_moments():
    u = inputs.uniform(0, 1, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3
    z = inputs.normal(0, 2, 200000)
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1) < 2e-2
    c = inputs.complex_normal(0, 3, 100000)
    assert abs(np.mean(np.abs(c) ** 2) - 1) < 2e-2


def test_beta22_law():
    x = inputs.beta22_points(0, 2, 100000) + 0.5
    assert x.min() >= 0 and x.max() < 1
    assert abs(x.mean() - 0.5) < 5e-3 and abs(x.var() - 0.05) < 2e-3  # Beta(2,2): var 1/20


def test_deterministic_and_offsets():
    a = inputs.uniform(7, 1, 10)
    b = inputs.uniform(7, 1, 20)
    assert np.array_equal(a, b[:10])
    assert np.array_equal(inputs.uniform(7, 1, 5, offset=5), b[5:10])
    assert not np.array_equal(inputs.uniform(7, 2, 10), a)


def test_workload_shapes():
    w = inputs.c1_small()
    assert w["x"].shape == (6, 2000) and len(w["terms"]) == 22
    assert np.all(w["x"] >= -0.5) and np.all(w["x"] < 0.5)
    w = inputs.c2_scale(M=1000)
    assert w["fhat"].size == 183851 and w["y"].size == 1000
