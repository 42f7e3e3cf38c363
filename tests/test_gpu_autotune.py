"""The plan autotuner: the chosen options meet the error target against the
FP64 oracle, the choice is the fastest candidate within the target, and a
target no candidate can meet is reported as unsupported."""
import numpy as np
import pytest

from oracle import anova, ndft
from paper_2010_10199_gb300 import inputs

from gpu_util import cplx_dev, f32_nodes, host, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gft():
    from paper_2010_10199_gb300 import build, gft as g
    build.build()
    g.load()
    return g


def test_autotune_choice_meets_target(gft):
    import torch
    x = inputs.uniform_points(31, 5, 20000)
    terms = anova.term_set(5, 2)
    bw = [0] + [16] * 5 + [8] * 10
    xd = to_dev(x, torch.float32)
    eps = 1e-5
    chosen, trials = gft.autotune(xd, terms, bw, eps=eps, reps=2)
    assert len(trials) >= 6
    ok = [t for t in trials if t["est_error"] <= eps]
    assert ok
    pick = [t for t in trials if t["chosen"]]
    assert len(pick) == 1
    assert pick[0]["ms_pair"] == min(t["ms_pair"] for t in ok)
    assert chosen["sigma"] == pick[0]["sigma"] and chosen["window_m_row"] == pick[0]["window_m_row"]
    assert len(trials) >= 8 and any(t["cell_kernel"] == 1 for t in trials)
    P = gft.Plan(xd, terms, bw, sigma=chosen["sigma"], window_m_row=chosen["window_m_row"],
                 n_ctas=chosen["n_ctas"], node_sort=chosen["node_sort"], cell_kernel=chosen["cell_kernel"])
    fhat = inputs.decaying_coefficients(2, terms, bw)
    y = inputs.complex_normal(2, 4, x.shape[1])
    xo = f32_nodes(x)
    ef = rel_l2(host(P.trafo(cplx_dev(fhat))), ndft.trafo(xo, terms, bw, fhat))
    eg = rel_l2(host(P.adjoint(cplx_dev(y))), ndft.adjoint(xo, terms, bw, y))
    # the estimate is the distance to a reference plan whose own error is far smaller
    assert max(ef, eg) <= 2 * eps, (ef, eg, chosen)


def test_autotune_unreachable_target(gft):
    import torch
    x = inputs.uniform_points(32, 3, 3000)
    terms = anova.term_set(3, 2)
    bw = [0, 16, 16, 16, 8, 8, 8]
    with pytest.raises(gft.AnovaError):
        gft.autotune(to_dev(x, torch.float32), terms, bw, eps=1e-13, reps=1)
