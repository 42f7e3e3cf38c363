"""The learned group screen: the network's kernels against the FP64 reference,
the screened path against plain FISTA, and what a trained network saves.

The screen has no counterpart in the paper; its result is pinned by
construction (every proposal is checked with the full KKT conditions), so the
screened path must reproduce plain full-group FISTA: the same active groups
and solutions within 1e-4 relative l2.
"""
import numpy as np
import pytest

from oracle import anova, mlp as omlp, solvers
from paper_2010_10199_gb300 import inputs

from gpu_util import cplx_dev, host, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gft():
    from paper_2010_10199_gb300 import build, gft as g
    build.build()
    g.load()
    return g


def _unpack(p, F, H):
    i = 0
    out = {}
    for k, shape in (("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, 1)), ("b3", (1,))):
        sz = int(np.prod(shape))
        out[k] = np.asarray(p[i:i + sz], dtype=np.float64).reshape(shape)
        i += sz
    return out


def _data(G=300, F=7, seed=3):
    X = inputs.normal(seed, 80, G * F).reshape(G, F)
    y = (inputs.uniform(seed, 81, G) < 0.2).astype(np.float64)
    return X, y


def test_mlp_forward_and_gradients_match_reference(gft):
    import torch
    F, H = 7, 128
    params = gft.mlp_init_params(5, F, H)
    net = gft.Mlp(params, F, H)
    X, y = _data()
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    ref_p = _unpack(params, F, H)
    X32 = X.astype(np.float32).astype(np.float64)
    cache = omlp.forward(ref_p, X32)
    prob = net.forward(Xd).cpu().numpy()
    assert np.max(np.abs(prob - cache["p"])) <= 1e-5
    loss = net.gradients(Xd, yd, pos_weight=2.5)
    assert abs(loss - omlp.loss(cache, y, 2.5)) <= 1e-5 * max(1.0, loss)
    _, g = net.params(grads=True)
    ref_g = omlp.backward(ref_p, cache, y, 2.5)
    got = _unpack(g, F, H)
    for k in omlp.PARAM_NAMES:
        err = np.linalg.norm(got[k] - ref_g[k]) / max(np.linalg.norm(ref_g[k]), 1e-30)
        assert err <= 1e-4, (k, err)
    net.close()


def test_adam_step_matches_reference(gft):
    import torch
    F, H = 7, 128
    params = gft.mlp_init_params(6, F, H)
    net = gft.Mlp(params, F, H)
    X, y = _data(G=200, seed=4)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    net.train(Xd, yd, batch=200, epochs=1, lr=1e-3, pos_weight=1.0)
    ref_p = _unpack(params, F, H)
    X32 = X.astype(np.float32).astype(np.float64)
    g = omlp.backward(ref_p, omlp.forward(ref_p, X32), y, 1.0)
    new = omlp.adam_step(ref_p, g, omlp.init_state(ref_p), lr=1e-3, step=1)
    got = _unpack(net.params(), F, H)
    for k in omlp.PARAM_NAMES:
        assert np.max(np.abs(got[k] - new[k])) <= 2e-6, k
    net.close()


def _problem(seed, d=10, M=5000):
    x = inputs.uniform_points(seed, d, M)
    terms = anova.term_set(d, 2)
    bw = [0] + [16] * d + [8] * (len(terms) - 1 - d)
    pairs = [tuple(sorted(inputs.choice(seed, inputs.S_CHOICE, d, 2, offset=8 * i))) for i in range(2)]
    single = [(inputs.choice(seed, inputs.S_CHOICE + 100, d, 1)[0],)]
    y = inputs.gaussian_bump_sum(x, pairs + single) + 0.02 * inputs.normal(seed, inputs.S_NOISE, M)
    return x, terms, bw, y.astype(np.complex128)


LAMS = list(np.geomspace(40.0, 6.0, 8))


def _active(path, terms, bw):
    offs, lens = anova.layout(terms, bw)
    return [solvers.group_norms(host(path[i]), offs, lens) > 0 for i in range(path.shape[0])]


def test_screened_path_equals_full_path(gft):
    import torch
    x, terms, bw, y = _problem(1)
    P = gft.Plan(to_dev(x, torch.float32), terms, bw)
    yd = cplx_dev(y)
    full, finfo, rc = P.fista(yd, LAMS, max_it=20000, tol=1e-8)
    assert rc == 0
    net = gft.Mlp(gft.mlp_init_params(9))   # untrained: correctness must not depend on the network
    scr, sinfo, stats = gft.fista_screened_path(P, net, yd, LAMS, max_it=20000, tol=1e-8, threshold=0.5)
    act_f, act_s = _active(full, terms, bw), _active(scr, terms, bw)
    for i in range(len(LAMS)):
        assert np.array_equal(act_f[i], act_s[i]), i
        assert rel_l2(host(scr[i]), host(full[i])) <= 1e-4, (i, rel_l2(host(scr[i]), host(full[i])))
    net.close()


def test_trained_screen_saves_transform_work(gft):
    """Train on the paths of four problems, screen three others: the screened
    paths transform a fraction of the terms the full paths do, with equal
    results.  Both paths stop at a relative change of 1e-6: an FP32 plan cannot
    resolve a relative change much below its resolution (2^-24, 6e-8), and at
    such a tolerance the iteration counts measure cycles at the rounding level
    (which differ between two paths of equal solutions) rather than work."""
    import torch
    Xs, ys = [], []
    for seed in (11, 12, 13, 14):
        x, terms, bw, y = _problem(seed)
        P = gft.Plan(to_dev(x, torch.float32), terms, bw)
        yd = cplx_dev(y)
        path, _, rc = P.fista(yd, LAMS, max_it=5000, tol=1e-6)
        X, lab = gft.screening_training_set(P, yd, LAMS, path)
        Xs.append(X)
        ys.append(lab)
        P.close()
    X = torch.cat(Xs).contiguous()
    lab = torch.cat(ys).contiguous()
    pos = float(lab.mean())
    net = gft.Mlp(gft.mlp_init_params(21))
    hist = net.train(X, lab, batch=256, epochs=150, lr=2e-3, pos_weight=max(1.0, (1 - pos) / max(pos, 1e-3)))
    assert hist[-1] < hist[0]
    fracs = []
    for seed in (2, 3, 4):
        x, terms, bw, y = _problem(seed)
        P = gft.Plan(to_dev(x, torch.float32), terms, bw)
        yd = cplx_dev(y)
        full, finfo, _ = P.fista(yd, LAMS, max_it=20000, tol=1e-6)
        scr, _, stats = gft.fista_screened_path(P, net, yd, LAMS, max_it=20000, tol=1e-6, threshold=0.5)
        for i in range(len(LAMS)):
            assert rel_l2(host(scr[i]), host(full[i])) <= 1e-4
        # transform work: terms transformed per iteration, summed over the path
        full_work = sum(fi["iterations"] for fi in finfo) * (len(terms) - 1)
        active = [int(a.sum()) for a in _active(full, terms, bw)]
        fracs.append(stats["term_iterations"] / full_work)
        print("problem", seed, "active groups per lambda", active, "screen stats", stats, "full work", full_work,
              "fraction", fracs[-1])
        P.close()
    assert np.mean(fracs) < 0.6 and max(fracs) < 0.7, fracs
    net.close()
