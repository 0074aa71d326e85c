"""The cost model's hand-written kernels (features, forward, masked-MSE
backward, Adam; through the C-ABI) against the float64 oracle in
oracle/mlp.py."""
import numpy as np
import pytest

from oracle import mlp
from paper_1706_10086_gb300 import inputs, tuning

pytestmark = pytest.mark.gpu


def to_list(flat, C):
    sizes = [(64, 7), (64,), (64, 64), (64,), (C, 64), (C,)]
    out, off = [], 0
    for s in sizes:
        n = int(np.prod(s))
        out.append(flat[off:off + n].astype(np.float64).reshape(s))
        off += n
    return out


def setup(C=9, B=37, seed=11):
    import torch
    flat = (inputs.uniform(seed, 0, (4672 + 65 * C,)) * 0.4).astype(np.float32)
    X = (inputs.uniform(seed + 1, 0, (B, 7)) * 2).astype(np.float32)
    T = inputs.uniform(seed + 2, 0, (B, C)).astype(np.float32)
    Mk = (inputs.uniform(seed + 3, 0, (B, C)) > -0.4).astype(np.float32)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return flat, X, T, Mk, d


def test_forward_matches_oracle(alp):
    import torch
    C, B = 9, 37
    flat, X, T, Mk, d = setup(C, B)
    Y = torch.empty(B, C, dtype=torch.float32, device="cuda")
    cache = torch.empty(B, 128, dtype=torch.float32, device="cuda")
    alp.alp_mlp_forward(d(flat), C, d(X), B, Y, cache)
    ref, (_, z1, _, z2, _) = mlp.forward(to_list(flat, C), X.astype(np.float64))
    assert np.allclose(Y.cpu().numpy(), ref, rtol=1e-5, atol=1e-5)
    c = cache.cpu().numpy()
    assert np.allclose(c[:, :64], z1, rtol=1e-5, atol=1e-5)
    assert np.allclose(c[:, 64:], z2, rtol=1e-5, atol=1e-5)


def test_backward_matches_oracle(alp):
    """GPU float32 gradients, element by element, within 1e-4 relative of the
    float64 backward pass (itself pinned by finite differences in the CPU
    tests), plus an absolute floor of 1e-5 of the tensor's largest gradient for
    elements whose contributions cancel to near zero (float32 sums over the
    batch carry about 1e-6 of the summands' magnitude)."""
    import torch
    C, B = 9, 37
    flat, X, T, Mk, d = setup(C, B)
    dP = d(flat)
    Y = torch.empty(B, C, dtype=torch.float32, device="cuda")
    cache = torch.empty(B, 128, dtype=torch.float32, device="cuda")
    grads = torch.empty(len(flat), dtype=torch.float32, device="cuda")
    work = torch.empty(B * (C + 128), dtype=torch.float32, device="cuda")
    loss = torch.zeros(2, dtype=torch.float32, device="cuda")
    alp.alp_mlp_forward(dP, C, d(X), B, Y, cache)
    alp.alp_mlp_backward(dP, C, d(X), B, cache, Y, d(T), d(Mk), grads, work, loss)
    P = to_list(flat, C)
    y, cch = mlp.forward(P, X.astype(np.float64))
    g_ref = mlp.backward(P, cch, y, T.astype(np.float64), Mk.astype(np.float64))
    g = to_list(grads.cpu().numpy(), C)
    names = ("W1", "b1", "W2", "b2", "W3", "b3")
    for name, a, b in zip(names, g, g_ref):
        tol = 1e-4 * np.abs(b) + 1e-5 * np.abs(b).max() + 1e-12
        bad = np.abs(a - b) > tol
        assert not bad.any(), (name, int(bad.sum()), float((np.abs(a - b) / tol).max()))
    assert abs(loss[0].item() - mlp.loss(y, T, Mk)) <= 1e-5 * mlp.loss(y, T, Mk)
    assert loss[1].item() == Mk.sum()


def test_adam_matches_oracle(alp):
    import torch
    n = 1000
    p = inputs.uniform(21, 0, (n,)).astype(np.float32)
    g = inputs.uniform(22, 0, (n,)).astype(np.float32)
    m = (inputs.uniform(23, 0, (n,)) * 0.1).astype(np.float32)
    v = (np.abs(inputs.uniform(24, 0, (n,))) * 0.01).astype(np.float32)
    d = lambda a: torch.from_numpy(a.copy()).cuda()
    dp, dm, dv = d(p), d(m), d(v)
    alp.alp_mlp_adam(dp, d(g), dm, dv, n, 7, 1e-2)
    rp, rm, rv = mlp.adam_step([p.astype(np.float64)], [g.astype(np.float64)],
                               [m.astype(np.float64)], [v.astype(np.float64)], 7, lr=1e-2)
    # float32 state and constants (1 - beta2 is 1.3e-5 off in float32): 1e-4 relative
    assert np.allclose(dp.cpu().numpy(), rp[0], rtol=1e-4, atol=1e-6)
    assert np.allclose(dm.cpu().numpy(), rm[0], rtol=1e-4, atol=1e-7)
    assert np.allclose(dv.cpu().numpy(), rv[0], rtol=1e-4, atol=1e-9)


def test_features_and_standardisation(alp):
    import torch
    sh = inputs.shapes(31, 50, 64, 16384)
    path = (np.arange(50) % 2).astype(np.int32)
    t = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    X = torch.empty(50, 7, dtype=torch.float32, device="cuda")
    alp.alp_mlp_features(50, t(sh[:, 0], torch.int64), t(sh[:, 1], torch.int64),
                         t(sh[:, 2], torch.int64), t(path, torch.int32), None, None, X)
    ref = mlp.features(sh[:, 0], sh[:, 1], sh[:, 2], path)
    assert np.allclose(X.cpu().numpy(), ref, rtol=1e-6, atol=1e-5)
    mean = torch.empty(7, dtype=torch.float32, device="cuda")
    std = torch.empty(7, dtype=torch.float32, device="cuda")
    alp.alp_mlp_feature_stats(50, X, mean, std)
    assert np.allclose(mean.cpu().numpy(), ref.mean(axis=0), rtol=1e-5, atol=1e-5)
    assert np.allclose(std.cpu().numpy(), ref.std(axis=0), rtol=1e-4, atol=1e-5)


def test_training_on_gpu_lowers_loss(alp):
    """A synthetic target with structure: the kernels' Adam loop fits it."""
    nat, emu = tuning.config_lists()
    C = len(nat) + len(emu)
    sh = inputs.shapes(41, 300, 64, 16384)
    path = (np.arange(300) % 2).astype(np.int32)
    lm = np.log2(sh).astype(np.float64)
    T = np.zeros((300, C))
    for c in range(C):
        T[:, c] = 0.1 * ((lm[:, 0] - 6 - (c % 9)) ** 2 % 7) + 0.05 * (c % 5) * path
    ds = {"M": sh[:, 0], "N": sh[:, 1], "K": sh[:, 2], "path": path,
          "T": T.astype(np.float32), "Mask": np.ones((300, C), np.float32), "C": C}
    model, hist = tuning.train(ds, epochs=400, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0], hist
