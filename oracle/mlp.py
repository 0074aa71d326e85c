"""Float64 reference of the tile-config cost model.  TEST INFRASTRUCTURE ONLY.

The model (a reading of the learned-predictor workload; the paper itself tunes
its tile size T by hand, Sect. 3 "Parameter Tuning" and Table 4):

    x  in R^7   standardised features of (M, N, K, path)
    h1 = relu(W1 x + b1)        W1: 64 x 7
    h2 = relu(W2 h1 + b2)       W2: 64 x 64
    y  = W3 h2 + b3             W3: C x 64, one output per tile configuration

    target  t_c = ln(time_c / best time of the shape), mask m_c = 1 where measured
    loss    L = sum_{n,c} m_nc (y_nc - t_nc)^2 / sum_{n,c} m_nc

Adam (Kingma and Ba, ICLR 2015) with bias correction:
    m = b1 m + (1-b1) g ;  v = b2 v + (1-b2) g^2
    w = w - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)

Every function is a direct transcription of these formulas in numpy float64.
"""
from __future__ import annotations

import numpy as np

NFEAT = 7
HIDDEN = 64


def features(M, N, K, path):
    """Raw (unstandardised) features: log2 M, log2 N, log2 K, log2(M/N),
    log2(N/K), log2(M/K), path flag (0 native, 1 emulated)."""
    M, N, K = (np.asarray(v, dtype=np.float64) for v in (M, N, K))
    lm, ln_, lk = np.log2(M), np.log2(N), np.log2(K)
    path = np.broadcast_to(np.asarray(path, dtype=np.float64), lm.shape)
    return np.stack([lm, ln_, lk, lm - ln_, ln_ - lk, lm - lk, path], axis=-1)


def forward(params, X):
    W1, b1, W2, b2, W3, b3 = params
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def loss(y, T, Mask):
    cnt = Mask.sum()
    return float((Mask * (y - T) ** 2).sum() / cnt)


def backward(params, cache, y, T, Mask):
    """Gradients of the masked MSE with respect to (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = params
    X, z1, h1, z2, h2 = cache
    cnt = Mask.sum()
    dy = 2.0 * Mask * (y - T) / cnt
    dW3 = dy.T @ h2
    db3 = dy.sum(axis=0)
    dh2 = dy @ W3
    dz2 = dh2 * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    dW1 = dz1.T @ X
    db1 = dz1.sum(axis=0)
    return [dW1, db1, dW2, db2, dW3, db3]


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for w, g, mm, vv in zip(params, grads, m, v):
        mm = b1 * mm + (1.0 - b1) * g
        vv = b2 * vv + (1.0 - b2) * g * g
        mhat = mm / (1.0 - b1 ** t)
        vhat = vv / (1.0 - b2 ** t)
        out_p.append(w - lr * mhat / (np.sqrt(vhat) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v


def numeric_grad(params, X, T, Mask, h=1e-6):
    """Central finite differences of the loss, one parameter at a time."""
    grads = []
    for pi, w in enumerate(params):
        g = np.zeros_like(w)
        it = np.nditer(w, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            saved = w[idx]
            w[idx] = saved + h
            lp = loss(forward(params, X)[0], T, Mask)
            w[idx] = saved - h
            lm = loss(forward(params, X)[0], T, Mask)
            w[idx] = saved
            g[idx] = (lp - lm) / (2.0 * h)
        grads.append(g)
    return grads
