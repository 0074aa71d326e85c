"""Helpers of the GPU tests: padded device matrices, oracle comparisons."""
import numpy as np


def dev(a, ld=None, pad_value=np.nan):
    """Row-major device copy of a 2-D array with leading dimension ``ld``
    (>= columns); the padding columns hold ``pad_value``."""
    import torch
    a = np.ascontiguousarray(a, dtype=np.float64)
    r, c = a.shape
    ld = c if ld is None else ld
    buf = np.full((max(r, 1), max(ld, 1)), pad_value)
    buf[:r, :c] = a
    return torch.from_numpy(buf).cuda(), ld


def host(t, r, c):
    return t.cpu().numpy()[:r, :c]


def assert_within_bound(got, ref, absAB, alpha, beta, C, K, U=2.0 ** -53, factor=1.0):
    bound = 2.0 * K * U * abs(alpha) * absAB
    if beta != 0.0:
        bound = bound + U * np.abs(beta * C)
    err = np.abs(got - ref)
    bad = err > factor * bound
    assert not np.isnan(got).any(), "NaN in result"
    assert not bad.any(), (f"{bad.sum()} entries out of bound; worst ratio "
                           f"{np.max(err / np.maximum(bound, 1e-300)):.3g}")
    return float(np.max(err / np.maximum(bound, 1e-300)))
