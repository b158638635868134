"""Pins the float64 MLP reference (oracle/mlp.py) to mathematics.

Gradients against central finite differences of the loss; the forward pass
in its affine regime against the composed affine map; the first Adam step
against its closed form (bias-corrected moments equal g and g^2).
"""
import numpy as np

from oracle import mlp


def small_params(seed):
    p = mlp.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.1
    p["b4"] = np.array([0.3])
    return p


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    p = small_params(3)
    x = rng.standard_normal((5, mlp.D_IN))
    t = rng.standard_normal(5)
    y, cache = mlp.forward(p, x)
    g = mlp.backward(p, cache, y, t)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        flat = p[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = mlp.loss(mlp.forward(p, x)[0], t)
            flat[i] = old - h
            lm = mlp.loss(mlp.forward(p, x)[0], t)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, an)


def test_forward_affine_regime():
    # positive weights, inputs and biases keep every ReLU open: the network is
    # the affine map x -> (w4^T W3 W2 W1) x + c
    rng = np.random.default_rng(4)
    p = {k: np.abs(v) for k, v in mlp.init_params(4).items()}
    for k in ("b1", "b2", "b3"):
        p[k] = np.abs(rng.standard_normal(p[k].shape))
    p["b4"] = np.array([0.25])
    x = np.abs(rng.standard_normal((7, mlp.D_IN)))
    y, _ = mlp.forward(p, x)
    row = ((p["w4"] @ p["W3"]) @ p["W2"]) @ p["W1"]
    c = p["w4"] @ (p["W3"] @ (p["W2"] @ p["b1"] + p["b2"]) + p["b3"]) + p["b4"][0]
    assert np.allclose(y, x @ row + c, rtol=1e-12, atol=1e-9)


def test_forward_dead_relu_gives_output_bias():
    p = mlp.init_params(5)
    p["b1"] = -1e6 * np.ones(mlp.D_H)     # every first-layer unit closed
    x = np.random.default_rng(5).standard_normal((3, mlp.D_IN))
    y, _ = mlp.forward(p, x)
    assert np.allclose(y, p["w4"] @ np.maximum(p["W3"] @ np.maximum(p["b2"], 0) + p["b3"], 0) + p["b4"][0])


def test_first_adam_step_closed_form():
    p = mlp.init_params(6)
    g = {k: np.random.default_rng(7).standard_normal(v.shape) for k, v in p.items()}
    before = {k: v.copy() for k, v in p.items()}
    lr, eps = 1e-3, 1e-8
    mlp.adam_step(p, g, {}, lr=lr, eps=eps)
    for k in p:
        assert np.allclose(p[k], before[k] - lr * g[k] / (np.abs(g[k]) + eps), rtol=0, atol=1e-15)
