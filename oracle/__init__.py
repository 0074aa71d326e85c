"""CPU oracle of the GEMM hot path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library (``paper_1706_10086_gb300``)
never does, and this package imports nothing from it: the two share no code.

Contents
--------
* ``alp_oracle.c`` (built here with gcc): the GEMM of Eq. 1 of Matthes et al.
  2017 as a long-double triple loop, ``|A||B|`` for the error bound, the
  emulated FP64 GEMM of the digit schemes (exponent scan, digit split in FP64
  steps, exact integer slice products, exact recombination rounded once to
  FP64) and its FP32 counterpart, and the modular scheme's definition (k-bit
  scaled integers, their exact product in 128-bit integers, one rounding; no
  residues or moduli).  Each is pinned in ``tests/test_oracle_pins.py``
  against exact rationals, derived bounds and integer cases.
* ``mlp.py``: the tile-config cost model (forward, backward, masked MSE, Adam)
  in float64 numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

BF16_DIGIT_BITS = 7     # b: bits per digit of the BF16-slice emulation


def build(force: bool = False) -> str:
    """Compiles ``alp_oracle.c`` into ``liboracle.so`` next to it."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            i64, f64, vp, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
            L.orc_gemm_f64.argtypes = [i64, i64, i64, f64, vp, i64, vp, i64, f64, vp, i64,
                                       vp, i64, vp, i64, i32]
            L.orc_absgemm.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, i64, i32]
            L.orc_row_exponents.argtypes = [i64, i64, vp, i64, vp]
            L.orc_col_exponents.argtypes = [i64, i64, vp, i64, vp]
            L.orc_split.argtypes = [i64, i64, vp, i64, vp, i32, i32, vp, vp]
            L.orc_emul_gemm.argtypes = [i64, i64, i64, f64, vp, i64, vp, i64, f64, vp, i64,
                                        vp, i64, i32, i32, i32, vp, i64, i32]
            L.orc_emul_gemm_f32.argtypes = L.orc_emul_gemm.argtypes
            L.orc_crt_gemm.argtypes = [i64, i64, i64, f64, vp, i64, vp, i64, f64, vp, i64, vp, i64,
                                       i32, vp, i64, i32]
            L.orc_int128_to_double.argtypes = [i64, ctypes.c_uint64]
            L.orc_int128_to_double.restype = ctypes.c_double
            for fn in ("orc_gemm_f64", "orc_absgemm", "orc_row_exponents", "orc_col_exponents",
                       "orc_split", "orc_emul_gemm", "orc_emul_gemm_f32", "orc_crt_gemm",
                       "orc_long_double_digits"):
                getattr(L, fn).restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _threads(nthreads):
    return nthreads if nthreads else (os.cpu_count() or 1)


def long_double_digits() -> int:
    return lib().orc_long_double_digits()


def gemm(alpha, A, B, beta, C=None, rows=None, nthreads=None):
    """``alpha*A@B + beta*C`` by the long-double triple loop (Eq. 1).

    ``rows``: optional row indices; the result then holds only those rows.
    ``C`` may be None when ``beta == 0`` (it is not read then)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    if C is None:
        C = np.zeros((M, N))
    C = _f64(C)
    ridx = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = M if ridx is None else len(ridx)
    D = np.empty((nr, N))
    rc = lib().orc_gemm_f64(M, N, K, float(alpha), _ptr(A), K, _ptr(B), N, float(beta),
                            _ptr(C), N, _ptr(D), N, _ptr(ridx), nr, _threads(nthreads))
    assert rc == 0
    return D


def absgemm(A, B, rows=None, nthreads=None):
    """``|A| @ |B|`` accumulated in long double (the magnitude in the error bound)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    N = B.shape[1]
    ridx = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = M if ridx is None else len(ridx)
    D = np.empty((nr, N))
    rc = lib().orc_absgemm(M, N, K, _ptr(A), K, _ptr(B), N, _ptr(D), N, _ptr(ridx), nr,
                           _threads(nthreads))
    assert rc == 0
    return D


def row_exponents(A):
    A = _f64(A)
    M, K = A.shape
    e = np.zeros(M, dtype=np.int32)
    bad = lib().orc_row_exponents(M, K, _ptr(A), K, _ptr(e))
    return e, bool(bad)


def col_exponents(B):
    B = _f64(B)
    K, N = B.shape
    f = np.zeros(N, dtype=np.int32)
    bad = lib().orc_col_exponents(K, N, _ptr(B), N, _ptr(f))
    return f, bool(bad)


def split(X, e, s, b=BF16_DIGIT_BITS):
    """Digits ``[s][R][K]`` (int32) and final remainders of a row-major matrix
    whose rows are scaled by ``2**-e``."""
    X = _f64(X)
    R, K = X.shape
    e = np.ascontiguousarray(e, dtype=np.int32)
    d = np.zeros((s, R, K), dtype=np.int32)
    rem = np.zeros((R, K))
    rc = lib().orc_split(R, K, _ptr(X), K, _ptr(e), s, b, _ptr(d), _ptr(rem))
    assert rc == 0
    return d, rem


def emul_gemm(alpha, A, B, beta, C, s, b=BF16_DIGIT_BITS, rows=None, nthreads=None, trim=False):
    """The emulated FP64 GEMM, bit-exact model of the GPU path.  ``trim``: the
    last group t = s+1 keeps only the pairs (1, s) and (s, 1).

    Returns (D, status): status 0 on success, 2 when A or B holds Inf/NaN."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    N = B.shape[1]
    if C is None:
        C = np.zeros((M, N))
    C = _f64(C)
    ridx = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = M if ridx is None else len(ridx)
    D = np.empty((nr, N))
    rc = lib().orc_emul_gemm(M, N, K, float(alpha), _ptr(A), K, _ptr(B), N, float(beta),
                             _ptr(C), N, _ptr(D), N, int(s), int(b), int(bool(trim)),
                             _ptr(ridx), nr,
                             _threads(nthreads))
    assert rc in (0, 2), rc
    return D, rc


def emul_gemm_f32(alpha, A, B, beta, C, s, b=8, rows=None, nthreads=None, trim=False):
    """The emulated GEMM for FP32 operands (float32 arrays, float alpha and
    beta), bit-exact model of the GPU's FP32 path.  Returns (D float32, status)."""
    A32, B32 = np.asarray(A, dtype=np.float32), np.asarray(B, dtype=np.float32)
    M, K = A32.shape
    N = B32.shape[1]
    C32 = np.zeros((M, N), np.float32) if C is None else np.asarray(C, dtype=np.float32)
    A64, B64, C64 = (_f64(x.astype(np.float64)) for x in (A32, B32, C32))
    ridx = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = M if ridx is None else len(ridx)
    D = np.empty((nr, N))
    rc = lib().orc_emul_gemm_f32(M, N, K, float(np.float32(alpha)), _ptr(A64), K, _ptr(B64), N,
                                 float(np.float32(beta)), _ptr(C64), N, _ptr(D), N, int(s), int(b),
                                 int(bool(trim)), _ptr(ridx), nr, _threads(nthreads))
    assert rc in (0, 2), rc
    return D.astype(np.float32), rc


def crt_gemm(alpha, A, B, beta, C, k, rows=None, nthreads=None):
    """The modular (CRT) emulated GEMM: the exact product of the operands
    rounded to k-bit integers per row and column, rounded once.  Returns
    (D, status)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    N = B.shape[1]
    if C is None:
        C = np.zeros((M, N))
    C = _f64(C)
    ridx = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = M if ridx is None else len(ridx)
    D = np.empty((nr, N))
    rc = lib().orc_crt_gemm(M, N, K, float(alpha), _ptr(A), K, _ptr(B), N, float(beta), _ptr(C),
                            N, _ptr(D), N, int(k), _ptr(ridx), nr, _threads(nthreads))
    assert rc in (0, 2), rc
    return D, rc


def int128_to_double(x: int) -> float:
    """The C oracle's conversion of a 128-bit integer to double."""
    x &= (1 << 128) - 1
    hi, lo = x >> 64, x & ((1 << 64) - 1)
    if hi >= 1 << 63:
        hi -= 1 << 64
    return lib().orc_int128_to_double(hi, lo)


U = 2.0 ** -53


def error_bound(alpha, absAB, beta, C, K):
    """Elementwise bound ``2 K u |alpha| (|A||B|)_ij + u |beta C_ij|`` (u = 2^-53)."""
    b = 2.0 * K * U * abs(alpha) * absAB
    if beta != 0.0 and C is not None:
        b = b + U * np.abs(beta * C)
    return b
