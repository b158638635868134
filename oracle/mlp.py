"""Float64 reference of the learned cost model (test infrastructure).

The paper has no learned component; this model is the project's surrogate
for the decompose search cost.  Definitions:

  layers   h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2),
           h3 = relu(h2 W3^T + b3), y = h3 w4 + b4
           x: (B, 64), W1: (256, 64), W2, W3: (256, 256), w4: (256,)
  loss     mean squared error 0.5 * mean((y - target)^2)
  update   Adam (Kingma & Ba, ICLR 2015) with bias correction

Every step here is a plain matrix product or an elementwise expression in
float64; the engine computes the same in BF16 operands / FP32 accumulation.
"""
from __future__ import annotations

import numpy as np

D_IN, D_H = 64, 256


def init_params(seed: int = 0, scale: float = 1.0):
    """He-style initialisation from a seeded numpy generator."""
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.standard_normal((D_H, D_IN)) * np.sqrt(2.0 / D_IN) * scale,
        "b1": np.zeros(D_H),
        "W2": rng.standard_normal((D_H, D_H)) * np.sqrt(2.0 / D_H) * scale,
        "b2": np.zeros(D_H),
        "W3": rng.standard_normal((D_H, D_H)) * np.sqrt(2.0 / D_H) * scale,
        "b3": np.zeros(D_H),
        "w4": rng.standard_normal(D_H) * np.sqrt(1.0 / D_H) * scale,
        "b4": np.zeros(1),
    }
    return p


def _id(a):
    return a


def forward(p, x, rnd=None):
    """y and the cached pre-activations / activations.

    rnd (optional) is applied to the hidden activations that feed the next
    product (h1, h2) -- the points where a low-precision engine stores its
    operands; None keeps everything in float64.
    """
    r = rnd or _id
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = r(np.maximum(z2, 0.0))
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = np.maximum(z3, 0.0)
    y = h3 @ p["w4"] + p["b4"][0]
    return y, {"x": x, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "z3": z3, "h3": h3}


def loss(y, target):
    d = np.asarray(y, dtype=np.float64) - np.asarray(target, dtype=np.float64)
    return 0.5 * float(np.mean(d * d))


def backward(p, cache, y, target, rnd=None):
    """Gradients of loss() with respect to every parameter.

    rnd (optional) is applied to dz3, dz2, dz1 where they feed a product
    (the bias gradients use the unrounded values).
    """
    r = rnd or _id
    B = y.shape[0]
    dy = (y - np.asarray(target, dtype=np.float64)) / B
    g = {}
    g["w4"] = cache["h3"].T @ dy
    g["b4"] = np.array([dy.sum()])
    dz3 = np.outer(dy, p["w4"]) * (cache["z3"] > 0)
    g["b3"] = dz3.sum(axis=0)
    dz3 = r(dz3)
    g["W3"] = dz3.T @ cache["h2"]
    dz2 = (dz3 @ p["W3"]) * (cache["z2"] > 0)
    g["b2"] = dz2.sum(axis=0)
    dz2 = r(dz2)
    g["W2"] = dz2.T @ cache["h1"]
    dz1 = (dz2 @ p["W2"]) * (cache["z1"] > 0)
    g["b1"] = dz1.sum(axis=0)
    dz1 = r(dz1)
    g["W1"] = dz1.T @ cache["x"]
    return g


def adam_step(p, g, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v and the step count."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] * g[k]
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return p
