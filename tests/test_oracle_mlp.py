"""Pins of the float64 cost-model reference (oracle/mlp.py): closed forms,
finite differences and the first-step property of Adam.  CPU-only."""
import numpy as np

from oracle import mlp
from paper_1706_10086_gb300 import inputs


def params(seed, C, scale=0.5):
    shapes = [(64, 7), (64,), (64, 64), (64,), (C, 64), (C,)]
    out, off = [], 0
    for shp in shapes:
        n = int(np.prod(shp))
        out.append(inputs.uniform(seed, off, shp) * scale)
        off += n
    return out


def test_zero_weights_give_bias():
    C = 5
    p = [np.zeros((64, 7)), np.zeros(64), np.zeros((64, 64)), np.zeros(64), np.zeros((C, 64)),
         np.arange(C, dtype=float)]
    X = inputs.uniform(1, 0, (3, 7))
    y, _ = mlp.forward(p, X)
    assert np.array_equal(y, np.tile(np.arange(C, dtype=float), (3, 1)))


def test_forward_single_path_closed_form():
    """Only unit 0 of each layer is wired: y = 2*relu(3*relu(x0 - 1)) + 0.5."""
    C = 1
    W1 = np.zeros((64, 7)); W1[0, 0] = 1.0
    b1 = np.zeros(64); b1[0] = -1.0
    W2 = np.zeros((64, 64)); W2[0, 0] = 3.0
    W3 = np.zeros((C, 64)); W3[0, 0] = 2.0
    p = [W1, b1, W2, np.zeros(64), W3, np.array([0.5])]
    x0 = np.array([-2.0, 0.5, 1.0, 1.25, 4.0])
    X = np.zeros((5, 7)); X[:, 0] = x0
    y, _ = mlp.forward(p, X)
    assert np.allclose(y[:, 0], 2 * np.maximum(3 * np.maximum(x0 - 1, 0), 0) + 0.5, rtol=0, atol=0)


def test_features():
    f = mlp.features(np.array([64]), np.array([256]), np.array([16]), 1)
    assert np.array_equal(f, [[6.0, 8.0, 4.0, -2.0, 4.0, 2.0, 1.0]])


def test_backward_matches_finite_differences():
    C = 4
    p = params(3, C)
    X = inputs.uniform(4, 0, (6, 7)) * 2
    T = inputs.uniform(5, 0, (6, C))
    Mask = (inputs.uniform(6, 0, (6, C)) > -0.3).astype(float)
    y, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, y, T, Mask)
    gn = mlp.numeric_grad(p, X, T, Mask, h=1e-6)
    for a, b in zip(g, gn):
        assert np.allclose(a, b, rtol=1e-5, atol=1e-8)


def test_adam_first_step_is_signed_lr():
    """With m = v = 0 and t = 1 the bias-corrected step is lr*g/(|g|+eps)."""
    w = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    z = [np.zeros(3)]
    p, m, v = mlp.adam_step(w, g, z, z, 1, lr=0.1)
    assert np.allclose(p[0], w[0] - 0.1 * g[0] / (np.abs(g[0]) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m[0], 0.1 * g[0]) and np.allclose(v[0], 0.001 * g[0] ** 2)


def test_training_lowers_loss_on_toy_set():
    C = 3
    p = params(8, C, scale=0.3)
    X = inputs.uniform(9, 0, (32, 7))
    T = np.stack([X[:, 0] ** 2, np.abs(X[:, 1]), X[:, 2] - X[:, 3]], axis=1)
    Mask = np.ones_like(T)
    m = [np.zeros_like(w) for w in p]
    v = [np.zeros_like(w) for w in p]
    l0 = mlp.loss(mlp.forward(p, X)[0], T, Mask)
    for t in range(1, 301):
        y, cache = mlp.forward(p, X)
        g = mlp.backward(p, cache, y, T, Mask)
        p, m, v = mlp.adam_step(p, g, m, v, t, lr=3e-3)
    l1 = mlp.loss(mlp.forward(p, X)[0], T, Mask)
    assert l1 < 0.2 * l0
