"""Pins of the FP64 screening-MLP reference: finite differences and a closed-form Adam step."""
import numpy as np

from oracle import mlp
from paper_2010_10199_gb300 import inputs


def _params(F=6, H=16, seed=0):
    def r(shape, s):
        return inputs.normal(seed, 40 + s, int(np.prod(shape))).reshape(shape) * 0.5
    return dict(W1=r((F, H), 1), b1=r((H,), 2), W2=r((H, H), 3), b2=r((H,), 4),
                W3=r((H, 1), 5), b3=r((1,), 6))


def test_gradients_match_central_differences():
    p = _params()
    X = inputs.normal(1, 50, 40 * 6).reshape(40, 6)
    y = (inputs.uniform(1, 51, 40) < 0.3).astype(np.float64)
    pw = 2.5
    g = mlp.backward(p, mlp.forward(p, X), y, pw)
    h = 1e-6
    for k in mlp.PARAM_NAMES:
        flat = p[k].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[i]
            flat[i] = old + h
            lp = mlp.loss(mlp.forward(p, X), y, pw)
            flat[i] = old - h
            lm = mlp.loss(mlp.forward(p, X), y, pw)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[i]) <= 1e-6 * max(1.0, abs(fd))


def test_first_adam_step_is_sign_step():
    # after one step m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    p = _params()
    X = inputs.normal(2, 50, 10 * 6).reshape(10, 6)
    y = np.array([1, 0, 0, 1, 0, 0, 0, 1, 0, 0], dtype=np.float64)
    g = mlp.backward(p, mlp.forward(p, X), y)
    q = mlp.adam_step(p, g, mlp.init_state(p), lr=1e-2, step=1)
    for k in mlp.PARAM_NAMES:
        assert np.allclose(p[k] - q[k], 1e-2 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-9, atol=1e-15)


def test_loss_is_stable_bce():
    p = _params()
    y = np.array([1.0, 0.0, 1.0, 0.0, 1.0])
    # moderate logits: equals the naive -[y log p + (1-y) log(1-p)]
    X = inputs.normal(3, 50, 5 * 6).reshape(5, 6)
    c = mlp.forward(p, X)
    ref = np.mean(-(y * np.log(c["p"]) + (1 - y) * np.log(1 - c["p"])))
    assert abs(mlp.loss(c, y) - ref) <= 1e-12 * max(1, ref)
    # huge logits: softplus(z) -> max(z, 0), so the loss is the mean of the wrong-side |z|
    c = mlp.forward(p, X * 1e4)
    z = c["z"]
    expect = np.mean(np.where(y > 0, np.maximum(-z, 0), np.maximum(z, 0)))
    assert np.isfinite(mlp.loss(c, y)) and abs(mlp.loss(c, y) - expect) <= 1e-9 * max(1, expect)
