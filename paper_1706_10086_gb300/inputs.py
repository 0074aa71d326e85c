"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module holds no GEMM arithmetic: it only turns a seed into numbers.  Both
the CUDA path and the CPU oracle receive the arrays it returns, so neither side
generates its own inputs.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in counter form: draw ``i`` of stream
``seed`` is ``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``, so any slice of the
stream can be produced without producing the ones before it.

Value maps (all vectorised with numpy, identical on x86_64 and aarch64):

* uniform in [-1, 1):   ``((x >> 11) * 2**-53) * 2 - 1``
* integers in {lo..hi}: ``lo + x % (hi - lo + 1)``
* emulation inputs:     ``u * 2**e``, ``u`` from draw 2n, ``e`` in [-phi, phi]
  from draw 2n+1 (the workload of the emulated-GEMM error study)
* log-uniform integers: ``round_half_even(exp(U(ln lo, ln hi)))`` clamped to
  [lo, hi], one draw per value.

Matrices of one problem share one stream: A takes draws [0, M*K), B the next
K*N and C the next M*N (twice as many per entry for the emulation inputs).
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Seed of each workload: 1706 + index of the workload in this list.
WORKLOADS = (
    "dgemm_512",          # plain DGEMM 512^3, alpha=1, beta=0 (+ integer variant)
    "dgemm_scan",         # native size scan 1024..16384, alpha=1.5, beta=0.5
    "emul_8192",          # emulated FP64 GEMM 8192^3, u*2^e inputs
    "batched_4096",       # 4096 variable-size problems, sizes log-uniform [16,1024]
    "mlp_predictor",      # tile-config predictor shapes, log-uniform [64,16384]
)


def workload_seed(name: str) -> int:
    return 1706 + WORKLOADS.index(name)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream ``seed``."""
    idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def to_uniform(x: np.ndarray) -> np.ndarray:
    """Maps 64-bit draws to doubles uniform in [-1, 1) (53 random bits)."""
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def to_int_range(x: np.ndarray, lo: int, hi: int) -> np.ndarray:
    return (x % np.uint64(hi - lo + 1)).astype(np.int64) + lo


def uniform(seed: int, start: int, shape) -> np.ndarray:
    n = int(np.prod(shape))
    return to_uniform(splitmix64(seed, start, n)).reshape(shape)


def integers(seed: int, start: int, shape, lo: int = -8, hi: int = 8) -> np.ndarray:
    n = int(np.prod(shape))
    return to_int_range(splitmix64(seed, start, n), lo, hi).astype(np.float64).reshape(shape)


def scaled(seed: int, start: int, shape, phi: int) -> np.ndarray:
    """Entries ``u * 2**e``: u uniform in [-1,1), e uniform integer in [-phi, phi]."""
    n = int(np.prod(shape))
    x = splitmix64(seed, 2 * start, 2 * n)
    u = to_uniform(x[0::2])
    e = to_int_range(x[1::2], -phi, phi)
    return np.ldexp(u, e.astype(np.int32)).reshape(shape)


def gemm_operands(seed: int, M: int, N: int, K: int, kind: str = "uniform", phi: int = 0,
                  with_c: bool = True):
    """Row-major A (MxK), B (KxN) and C (MxN) of one problem from one stream.

    ``kind`` is "uniform" ([-1,1)), "int" ({-8..8}) or "scaled" (u*2^e, exponent
    range ``phi``; C, when asked for, is then uniform).
    """
    sizes = (M * K, K * N, M * N)
    offs = (0, sizes[0], sizes[0] + sizes[1])
    if kind == "uniform":
        gen = lambda off, shp: uniform(seed, off, shp)
    elif kind == "int":
        gen = lambda off, shp: integers(seed, off, shp)
    elif kind == "scaled":
        gen = lambda off, shp: scaled(seed, off, shp, phi)
    else:
        raise ValueError(kind)
    A = gen(offs[0], (M, K))
    B = gen(offs[1], (K, N))
    if not with_c:
        return A, B, None
    C = uniform(seed, offs[2] * (2 if kind == "scaled" else 1), (M, N)) if kind == "scaled" \
        else gen(offs[2], (M, N))
    return A, B, C


def log_uniform_ints(seed: int, start: int, count: int, lo: int, hi: int) -> np.ndarray:
    u = (splitmix64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    v = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    return np.clip(np.rint(v), lo, hi).astype(np.int64)


def shapes(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """``count`` (M, N, K) triples, each entry log-uniform in [lo, hi]."""
    return log_uniform_ints(seed, 0, 3 * count, lo, hi).reshape(count, 3)
