"""FP64 reference of the group-screening MLP (oracle; test infrastructure only).

The paper has no learned component; this network is an addition that proposes
which ANOVA groups are active along a group-lasso lambda path.  Its labels are
the method's own active sets: the groups u with f_u != 0 at the solution of
eq. (alligatoah), Sec. 4.2.  The reference below is the textbook two-hidden-
layer perceptron; the CUDA forward/backward kernels are checked against it.

    h1 = relu(X W1 + b1)          X: [G, F], W1: [F, H]
    h2 = relu(h1 W2 + b2)         W2: [H, H]
    z  = h2 W3 + b3               W3: [H, 1]
    p  = sigmoid(z)
    loss = mean_g [ pw * y_g * softplus(-z_g) + (1 - y_g) * softplus(z_g) ]

(binary cross-entropy on logits with a positive-class weight ``pw``) and one
Adam step (Kingma and Ba, 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def softplus(z):
    return np.logaddexp(0.0, z)


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def forward(params: dict, X: np.ndarray) -> dict:
    a1 = X @ params["W1"] + params["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ params["W2"] + params["b2"]
    h2 = np.maximum(a2, 0.0)
    z = (h2 @ params["W3"] + params["b3"]).reshape(-1)
    return dict(X=X, a1=a1, h1=h1, a2=a2, h2=h2, z=z, p=sigmoid(z))


def loss(cache: dict, y: np.ndarray, pw: float = 1.0) -> float:
    z = cache["z"]
    return float(np.mean(pw * y * softplus(-z) + (1.0 - y) * softplus(z)))


def backward(params: dict, cache: dict, y: np.ndarray, pw: float = 1.0) -> dict:
    G = y.size
    z = cache["z"]
    s = sigmoid(z)
    dz = ((1.0 - y) * s - pw * y * (1.0 - s)) / G           # d loss / d z
    dW3 = cache["h2"].T @ dz[:, None]
    db3 = np.array([dz.sum()])
    dh2 = dz[:, None] @ params["W3"].T
    da2 = dh2 * (cache["a2"] > 0)
    dW2 = cache["h1"].T @ da2
    db2 = da2.sum(axis=0)
    dh1 = da2 @ params["W2"].T
    da1 = dh1 * (cache["a1"] > 0)
    dW1 = cache["X"].T @ da1
    db1 = da1.sum(axis=0)
    return dict(W1=dW1, b1=db1, W2=dW2, b2=db2, W3=dW3, b3=db3)


def adam_step(params: dict, grads: dict, state: dict, lr: float, beta1=0.9, beta2=0.999,
              eps=1e-8, step: int = 1) -> dict:
    """One Adam update (m, v moments with bias correction); returns new params."""
    out = {}
    for k in PARAM_NAMES:
        m = beta1 * state[k + "_m"] + (1 - beta1) * grads[k]
        v = beta2 * state[k + "_v"] + (1 - beta2) * grads[k] ** 2
        state[k + "_m"], state[k + "_v"] = m, v
        mh = m / (1 - beta1 ** step)
        vh = v / (1 - beta2 ** step)
        out[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return out


def init_state(params: dict) -> dict:
    st = {}
    for k in PARAM_NAMES:
        st[k + "_m"] = np.zeros_like(params[k])
        st[k + "_v"] = np.zeros_like(params[k])
    return st
