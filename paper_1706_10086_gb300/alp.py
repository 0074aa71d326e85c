"""Python binding of the C-ABI in ``include/alp.h`` / ``include/alp_ext.h``.

Argument marshalling only: every function forwards to the ``extern "C"`` entry
point of the same name in ``libalp.so`` (built from ``csrc/`` for sm_103a).
Device buffers may be given as torch CUDA tensors (their ``data_ptr()`` is
passed) or as raw integer addresses; ``stream`` is a ``torch.cuda.Stream``, a
raw ``cudaStream_t`` integer, or None for the current torch stream.  There is
no fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libalp.so")

# alp_status
ALP_OK = 0
ALP_ERR_INVALID_ARG = 1
ALP_ERR_UNSUPPORTED = 2
ALP_ERR_CUDA = 3
ALP_ERR_TIMEOUT = 4
ALP_ERR_WORKSPACE = 5
ALP_ERR_NOT_TUNED = 6
# alp_slice_kind
ALP_SLICE_INT8 = 0
ALP_SLICE_BF16 = 1
ALP_SLICE_BF16_B8 = 2
ALP_SLICE_BF16_B8_TRIM = 3
ALP_SLICE_BF16_CRT = 4
# alp_path
ALP_PATH_NATIVE = 0
ALP_PATH_EMUL = 1
# alp_tune_mode
ALP_TUNE_EXHAUSTIVE = 0
ALP_TUNE_PREDICT = 1
ALP_TUNE_LOOKUP = 2


class alp_config(ctypes.Structure):
    _fields_ = [("bm", ctypes.c_int32), ("bn", ctypes.c_int32), ("bk", ctypes.c_int32),
                ("tm", ctypes.c_int32), ("tn", ctypes.c_int32), ("stages", ctypes.c_int32)]

    def astuple(self):
        return (self.bm, self.bn, self.bk, self.tm, self.tn, self.stages)

    def __repr__(self):
        return "alp_config(bm=%d, bn=%d, bk=%d, tm=%d, tn=%d, stages=%d)" % self.astuple()


class AlpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)}")


_lock = threading.Lock()
_lib = None

_i64, _f64, _vp, _int = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
_f32 = ctypes.c_float
_SIGS = {
    "alp_status_string": ([_int], ctypes.c_char_p),
    "alp_gemm_f64": ([_i64, _i64, _i64, _f64, _vp, _i64, _vp, _i64, _f64, _vp, _i64,
                      ctypes.POINTER(alp_config), _vp], _int),
    "alp_gemm_f64_emul": ([_i64, _i64, _i64, _f64, _vp, _i64, _vp, _i64, _f64, _vp, _i64,
                           _int, _int, _vp, ctypes.c_size_t, _vp], _int),
    "alp_gemm_f64_emul_workspace": ([_i64, _i64, _i64, _int, _int], ctypes.c_size_t),
    "alp_emul_exponents": ([_i64, _i64, _vp, _i64, _int, _vp, _vp], _int),
    "alp_emul_split": ([_i64, _i64, _vp, _i64, _int, _vp, _int, _int, _vp, _i64, _vp], _int),
    "alp_emul_scan_split_rows": ([_i64, _i64, _vp, _i64, _vp, _int, _int, _vp, _i64, _vp], _int),
    "alp_emul_slice_products": ([_i64, _i64, _i64, _int, _int, _vp, _vp, _i64, _vp, _i64, _vp],
                                _int),
    "alp_emul_recombine": ([_i64, _i64, _int, _int, _vp, _i64, _vp, _vp, _f64, _f64, _vp, _i64,
                            _vp],
                           _int),
    "alp_emul_crt_bits": ([_i64, _int], _int),
    "alp_emul_crt_choose": ([_int, _int, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp,
                             ctypes.c_size_t, _vp, ctypes.POINTER(_int), ctypes.POINTER(_f64)],
                            _int),
    "alp_emul_crt_moduli_rule": ([_i64, _i64, _i64, ctypes.POINTER(_f64), ctypes.POINTER(_f64)],
                                 _int),
    "alp_emul_recombine_crt": ([_i64, _i64, _i64, _int, _vp, _i64, _vp, _vp, _f64, _f64, _vp,
                                _i64, _vp], _int),
    "alp_emul_products_recombine_crt": ([_i64, _i64, _i64, _int, _vp, _vp, _i64, _vp, _i64,
                                         _vp, _vp, _f64, _f64, _vp, _i64, _vp, ctypes.c_size_t,
                                         _vp], _int),
    "alp_emul_products_recombine_crt_workspace": ([_i64, _i64], ctypes.c_size_t),
    "alp_gemm_f32_emul": ([_i64, _i64, _i64, _f32, _vp, _i64, _vp, _i64, _f32, _vp, _i64, _int,
                           _int, _vp, ctypes.c_size_t, _vp], _int),
    "alp_gemm_f32_emul_workspace": ([_i64, _i64, _i64, _int, _int], ctypes.c_size_t),
    "alp_host_access": ([ctypes.POINTER(_int), ctypes.POINTER(_int)], _int),
    "alp_gemm_f64_ex": ([_int, _int, _i64, _i64, _i64, _f64, _vp, _i64, _vp, _i64, _f64, _vp,
                         _i64, ctypes.POINTER(alp_config), _vp, ctypes.c_size_t, _vp], _int),
    "alp_gemm_f64_ex_workspace": ([_int, _int, _i64, _i64, _i64], ctypes.c_size_t),
    "alp_gemm_f64_emul_ex": ([_int, _int, _i64, _i64, _i64, _f64, _vp, _i64, _vp, _i64, _f64, _vp,
                              _i64, _int, _int, _vp, ctypes.c_size_t, _vp], _int),
    "alp_gemm_f32_emul_ex": ([_int, _int, _i64, _i64, _i64, _f32, _vp, _i64, _vp, _i64, _f32, _vp,
                              _i64, _int, _int, _vp, ctypes.c_size_t, _vp], _int),
    "alp_gemm_f64_cm": ([_int, _int, _i64, _i64, _i64, _f64, _vp, _i64, _vp, _i64, _f64, _vp,
                         _i64, ctypes.POINTER(alp_config), _vp, ctypes.c_size_t, _vp], _int),
    "alp_gemm_f64_cm_workspace": ([_int, _int, _i64, _i64, _i64], ctypes.c_size_t),
    "alp_gemm_f64_emul_cm": ([_int, _int, _i64, _i64, _i64, _f64, _vp, _i64, _vp, _i64, _f64, _vp,
                              _i64, _int, _int, _vp, ctypes.c_size_t, _vp], _int),
    "alp_gemm_f64_emul_cm_workspace": ([_i64, _i64, _i64, _int, _int], ctypes.c_size_t),
    "alp_gemm_f32_emul_cm": ([_int, _int, _i64, _i64, _i64, _f32, _vp, _i64, _vp, _i64, _f32, _vp,
                              _i64, _int, _int, _vp, ctypes.c_size_t, _vp], _int),
    "alp_gemm_f32_emul_cm_workspace": ([_i64, _i64, _i64, _int, _int], ctypes.c_size_t),
    "alp_emul_exponents_f32": ([_i64, _i64, _vp, _i64, _int, _vp, _vp], _int),
    "alp_emul_split_f32": ([_i64, _i64, _vp, _i64, _int, _vp, _int, _int, _vp, _i64, _vp], _int),
    "alp_emul_recombine_f32": ([_i64, _i64, _int, _int, _vp, _i64, _vp, _vp, _f32, _f32, _vp, _i64,
                                _vp], _int),
    "alp_gemm_batched_varsize": ([_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                  _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp], _int),
    "alp_gemm_batched_workspace": ([_i64, _vp, _vp, _vp], ctypes.c_size_t),
    "alp_tune": ([_i64, _i64, _i64, _int, _int, ctypes.POINTER(alp_config),
                  ctypes.POINTER(_f64)], _int),
    "alp_get_device_error": ([_vp], _int),
    "alp_config_valid": ([ctypes.POINTER(alp_config), _int], _int),
    "alp_config_smem_bytes": ([ctypes.POINTER(alp_config)], _i64),
    "alp_config_threads": ([ctypes.POINTER(alp_config)], _int),
    "alp_config_count": ([_int], _int),
    "alp_config_at": ([_int, _int, ctypes.POINTER(alp_config)], _int),
    "alp_set_wait_timeout_ms": ([_f64], _int),
    "alp_debug_inject_skip": ([_int], _int),
    "alp_probe_fp64_peak": ([_int, _i64, _int, _int, ctypes.POINTER(_f64), _vp], _int),
    "alp_emul_tail_split": ([_int, _int, _int, _int, ctypes.POINTER(_int), ctypes.POINTER(_int),
                             ctypes.POINTER(_int), ctypes.POINTER(_int)], _int),
    "alp_tune_time_config": ([_i64, _i64, _i64, _int, ctypes.POINTER(alp_config), _int, _int,
                              ctypes.POINTER(_f64)], _int),
    "alp_tune_set_cached": ([_i64, _i64, _i64, _int, ctypes.POINTER(alp_config)], _int),
    "alp_tune_clear_cache": ([], _int),
    "alp_mlp_param_count": ([_int], _i64),
    "alp_mlp_features": ([_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _int),
    "alp_mlp_feature_stats": ([_i64, _vp, _vp, _vp, _vp], _int),
    "alp_mlp_forward": ([_vp, _int, _vp, _i64, _vp, _vp, _vp], _int),
    "alp_mlp_backward": ([_vp, _int, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _int),
    "alp_mlp_adam": ([_vp, _vp, _vp, _vp, _i64, _int, ctypes.c_float, ctypes.c_float,
                      ctypes.c_float, ctypes.c_float, _vp], _int),
    "alp_tune_load_model": ([_vp, _int, _vp, _vp], _int),
    "alp_tune_unload_model": ([], _int),
    "alp_batched_class_of": ([_i64, _i64], _int),
    "alp_batched_set_class_config": ([_int, _int, _int, _int], _int),
    "alp_batched_get_class_config": ([_int, ctypes.POINTER(_int), ctypes.POINTER(_int),
                                      ctypes.POINTER(_int)], _int),
    "alp_batched_graph_create": ([_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                  _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                  ctypes.POINTER(_vp)], _int),
    "alp_batched_graph_launch": ([_vp, _vp], _int),
    "alp_gemm_batched_varsize_noalloc": ([_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                          _vp, _vp, _vp, _vp, _vp, _vp], _int),
    "alp_batched_graph_destroy": ([_vp], _int),
}


def lib():
    """The loaded ``libalp.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                                   "(the CUDA library is required; there is no fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def exported_symbols():
    """Names of _SIGS found in the library."""
    L = lib()
    return [n for n in _SIGS if getattr(L, n, None) is not None]


def _p(x):
    """Device address of a torch tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _s(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, where: str, raise_on_error: bool):
    if raise_on_error and status != ALP_OK:
        raise AlpError(status, where)
    return status


def status_string(status: int) -> str:
    return lib().alp_status_string(int(status)).decode()


def alp_gemm_f64(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cfg=None, stream=None,
                 raise_on_error=True):
    c = None
    if cfg is not None:
        c = cfg if isinstance(cfg, alp_config) else alp_config(*cfg)
    st = lib().alp_gemm_f64(M, N, K, float(alpha), _p(A), lda, _p(B), ldb, float(beta), _p(C),
                            ldc, ctypes.byref(c) if c is not None else None, _s(stream))
    return _check(st, "alp_gemm_f64", raise_on_error)


def alp_host_access():
    """(pageable, host_page_tables) of the current device (see alp_ext.h)."""
    a, b = _int(0), _int(0)
    _check(lib().alp_host_access(ctypes.byref(a), ctypes.byref(b)), "alp_host_access", True)
    return a.value, b.value


def alp_gemm_f64_ex(trans_a, trans_b, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cfg=None,
                    workspace=None, workspace_bytes=0, stream=None, raise_on_error=True):
    c = None
    if cfg is not None:
        c = cfg if isinstance(cfg, alp_config) else alp_config(*cfg)
    st = lib().alp_gemm_f64_ex(int(trans_a), int(trans_b), M, N, K, float(alpha), _p(A), lda,
                               _p(B), ldb, float(beta), _p(C), ldc,
                               ctypes.byref(c) if c is not None else None, _p(workspace),
                               int(workspace_bytes), _s(stream))
    return _check(st, "alp_gemm_f64_ex", raise_on_error)


def alp_gemm_f64_ex_workspace(trans_a, trans_b, M, N, K):
    return int(lib().alp_gemm_f64_ex_workspace(int(trans_a), int(trans_b), M, N, K))


def alp_gemm_f64_emul(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nslices, kind, workspace,
                      workspace_bytes, stream=None, raise_on_error=True):
    st = lib().alp_gemm_f64_emul(M, N, K, float(alpha), _p(A), lda, _p(B), ldb, float(beta),
                                 _p(C), ldc, int(nslices), int(kind), _p(workspace),
                                 int(workspace_bytes), _s(stream))
    return _check(st, "alp_gemm_f64_emul", raise_on_error)


def alp_gemm_f64_emul_workspace(M, N, K, nslices, kind=ALP_SLICE_BF16):
    return int(lib().alp_gemm_f64_emul_workspace(M, N, K, int(nslices), int(kind)))


def alp_emul_exponents(rows, cols, X, ldx, trans, exps, stream=None, raise_on_error=True):
    st = lib().alp_emul_exponents(rows, cols, _p(X), ldx, int(trans), _p(exps), _s(stream))
    return _check(st, "alp_emul_exponents", raise_on_error)


def alp_emul_split(R, K, X, ldx, trans, exps, nslices, kind, out, kpad, stream=None,
                   raise_on_error=True):
    st = lib().alp_emul_split(R, K, _p(X), ldx, int(trans), _p(exps), int(nslices), int(kind),
                              _p(out), kpad, _s(stream))
    return _check(st, "alp_emul_split", raise_on_error)


def alp_emul_scan_split_rows(R, K, X, ldx, exps, nslices, kind, out, kpad, stream=None,
                             raise_on_error=True):
    st = lib().alp_emul_scan_split_rows(R, K, _p(X), ldx, _p(exps), int(nslices), int(kind),
                                        _p(out), kpad, _s(stream))
    return _check(st, "alp_emul_scan_split_rows", raise_on_error)


def alp_emul_slice_products(M, N, K, nslices, kind, da, db, kpad, G, ldg, stream=None,
                            raise_on_error=True):
    st = lib().alp_emul_slice_products(M, N, K, int(nslices), int(kind), _p(da), _p(db), kpad,
                                       _p(G), ldg, _s(stream))
    return _check(st, "alp_emul_slice_products", raise_on_error)


def alp_emul_recombine(M, N, nslices, kind, G, ldg, e, f, alpha, beta, C, ldc, stream=None,
                       raise_on_error=True):
    st = lib().alp_emul_recombine(M, N, int(nslices), int(kind), _p(G), ldg, _p(e), _p(f),
                                  float(alpha), float(beta), _p(C), ldc, _s(stream))
    return _check(st, "alp_emul_recombine", raise_on_error)


def alp_emul_crt_bits(K, nmoduli):
    return int(lib().alp_emul_crt_bits(K, int(nmoduli)))


def alp_emul_crt_choose(trans_a, trans_b, M, N, K, A, lda, B, ldb, workspace, workspace_bytes,
                        stream=None, raise_on_error=True):
    """The automatic modulus count for op(A) op(B) (one stream synchronisation).
    Returns (count, (predicted componentwise error in units of 2^-53,
    predicted normwise ratio to native))."""
    n = _int(0)
    pred = (_f64 * 2)()
    st = lib().alp_emul_crt_choose(int(trans_a), int(trans_b), M, N, K, _p(A), lda, _p(B), ldb,
                                   _p(workspace), workspace_bytes, _s(stream), ctypes.byref(n),
                                   pred)
    _check(st, "alp_emul_crt_choose", raise_on_error)
    return n.value, (pred[0], pred[1])


def alp_emul_crt_moduli_rule(M, N, K, stats):
    """The automatic-count rule on given statistics (host only).  Returns
    (count, (componentwise prediction, normwise ratio))."""
    st = (_f64 * 6)(*[float(v) for v in stats])
    pred = (_f64 * 2)()
    n = lib().alp_emul_crt_moduli_rule(M, N, K, st, pred)
    return int(n), (pred[0], pred[1])


def alp_emul_recombine_crt(M, N, K, nmoduli, G, ldg, e, f, alpha, beta, C, ldc, stream=None,
                           raise_on_error=True):
    st = lib().alp_emul_recombine_crt(M, N, K, int(nmoduli), _p(G), ldg, _p(e), _p(f),
                                      float(alpha), float(beta), _p(C), ldc, _s(stream))
    return _check(st, "alp_emul_recombine_crt", raise_on_error)


def alp_emul_products_recombine_crt_workspace(M, N):
    return int(lib().alp_emul_products_recombine_crt_workspace(M, N))


def alp_emul_products_recombine_crt(M, N, K, nmoduli, da, db, kpad, G, ldg, e, f, alpha, beta, C,
                                    ldc, workspace=None, workspace_bytes=0, stream=None,
                                    raise_on_error=True):
    st = lib().alp_emul_products_recombine_crt(M, N, K, int(nmoduli), _p(da), _p(db), kpad,
                                               _p(G), ldg, _p(e), _p(f), float(alpha),
                                               float(beta), _p(C), ldc, _p(workspace),
                                               int(workspace_bytes), _s(stream))
    return _check(st, "alp_emul_products_recombine_crt", raise_on_error)


def alp_gemm_f32_emul(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nslices,
                      kind=ALP_SLICE_BF16_B8, workspace=None, workspace_bytes=0, stream=None,
                      raise_on_error=True):
    st = lib().alp_gemm_f32_emul(M, N, K, float(alpha), _p(A), lda, _p(B), ldb, float(beta),
                                 _p(C), ldc, int(nslices), int(kind), _p(workspace),
                                 int(workspace_bytes), _s(stream))
    return _check(st, "alp_gemm_f32_emul", raise_on_error)


def alp_gemm_f32_emul_workspace(M, N, K, nslices, kind=ALP_SLICE_BF16_B8):
    return int(lib().alp_gemm_f32_emul_workspace(M, N, K, int(nslices), int(kind)))


def alp_gemm_f64_emul_ex(trans_a, trans_b, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                         nslices, kind=ALP_SLICE_BF16, workspace=None, workspace_bytes=0,
                         stream=None, raise_on_error=True):
    st = lib().alp_gemm_f64_emul_ex(int(trans_a), int(trans_b), M, N, K, float(alpha), _p(A), lda,
                                    _p(B), ldb, float(beta), _p(C), ldc, int(nslices), int(kind),
                                    _p(workspace), int(workspace_bytes), _s(stream))
    return _check(st, "alp_gemm_f64_emul_ex", raise_on_error)


def alp_gemm_f32_emul_ex(trans_a, trans_b, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                         nslices, kind=ALP_SLICE_BF16_B8, workspace=None, workspace_bytes=0,
                         stream=None, raise_on_error=True):
    st = lib().alp_gemm_f32_emul_ex(int(trans_a), int(trans_b), M, N, K, float(alpha), _p(A), lda,
                                    _p(B), ldb, float(beta), _p(C), ldc, int(nslices), int(kind),
                                    _p(workspace), int(workspace_bytes), _s(stream))
    return _check(st, "alp_gemm_f32_emul_ex", raise_on_error)


def alp_gemm_f64_cm(trans_a, trans_b, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cfg=None,
                    workspace=None, workspace_bytes=0, stream=None, raise_on_error=True):
    c = None
    if cfg is not None:
        c = cfg if isinstance(cfg, alp_config) else alp_config(*cfg)
    st = lib().alp_gemm_f64_cm(int(trans_a), int(trans_b), M, N, K, float(alpha), _p(A), lda,
                               _p(B), ldb, float(beta), _p(C), ldc,
                               ctypes.byref(c) if c is not None else None, _p(workspace),
                               int(workspace_bytes), _s(stream))
    return _check(st, "alp_gemm_f64_cm", raise_on_error)


def alp_gemm_f64_cm_workspace(trans_a, trans_b, M, N, K):
    return int(lib().alp_gemm_f64_cm_workspace(int(trans_a), int(trans_b), M, N, K))


def alp_gemm_f64_emul_cm(trans_a, trans_b, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                         nslices, kind=ALP_SLICE_BF16_CRT, workspace=None, workspace_bytes=0,
                         stream=None, raise_on_error=True):
    st = lib().alp_gemm_f64_emul_cm(int(trans_a), int(trans_b), M, N, K, float(alpha), _p(A), lda,
                                    _p(B), ldb, float(beta), _p(C), ldc, int(nslices), int(kind),
                                    _p(workspace), int(workspace_bytes), _s(stream))
    return _check(st, "alp_gemm_f64_emul_cm", raise_on_error)


def alp_gemm_f64_emul_cm_workspace(M, N, K, nslices, kind):
    return int(lib().alp_gemm_f64_emul_cm_workspace(M, N, K, int(nslices), int(kind)))


def alp_gemm_f32_emul_cm(trans_a, trans_b, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                         nslices, kind=ALP_SLICE_BF16_B8, workspace=None, workspace_bytes=0,
                         stream=None, raise_on_error=True):
    st = lib().alp_gemm_f32_emul_cm(int(trans_a), int(trans_b), M, N, K, float(alpha), _p(A), lda,
                                    _p(B), ldb, float(beta), _p(C), ldc, int(nslices), int(kind),
                                    _p(workspace), int(workspace_bytes), _s(stream))
    return _check(st, "alp_gemm_f32_emul_cm", raise_on_error)


def alp_gemm_f32_emul_cm_workspace(M, N, K, nslices, kind):
    return int(lib().alp_gemm_f32_emul_cm_workspace(M, N, K, int(nslices), int(kind)))


def alp_emul_exponents_f32(rows, cols, X, ldx, trans, exps, stream=None, raise_on_error=True):
    st = lib().alp_emul_exponents_f32(rows, cols, _p(X), ldx, int(trans), _p(exps), _s(stream))
    return _check(st, "alp_emul_exponents_f32", raise_on_error)


def alp_emul_split_f32(R, K, X, ldx, trans, exps, nslices, kind, out, kpad, stream=None,
                       raise_on_error=True):
    st = lib().alp_emul_split_f32(R, K, _p(X), ldx, int(trans), _p(exps), int(nslices),
                                  int(kind), _p(out), kpad, _s(stream))
    return _check(st, "alp_emul_split_f32", raise_on_error)


def alp_emul_recombine_f32(M, N, nslices, kind, G, ldg, e, f, alpha, beta, C, ldc, stream=None,
                           raise_on_error=True):
    st = lib().alp_emul_recombine_f32(M, N, int(nslices), int(kind), _p(G), ldg, _p(e), _p(f),
                                      float(alpha), float(beta), _p(C), ldc, _s(stream))
    return _check(st, "alp_emul_recombine_f32", raise_on_error)


def alp_gemm_batched_varsize(count, dM, dN, dK, dalpha, dA, dlda, dB, dldb, dbeta, dC, dldc,
                             hM, hN, hK, workspace, workspace_bytes, stream=None,
                             raise_on_error=True):
    st = lib().alp_gemm_batched_varsize(count, _p(dM), _p(dN), _p(dK), _p(dalpha), _p(dA),
                                        _p(dlda), _p(dB), _p(dldb), _p(dbeta), _p(dC),
                                        _p(dldc), _host(hM), _host(hN), _host(hK),
                                        _p(workspace), int(workspace_bytes), _s(stream))
    return _check(st, "alp_gemm_batched_varsize", raise_on_error)


def alp_gemm_batched_workspace(count, hM, hN, hK):
    return int(lib().alp_gemm_batched_workspace(count, _host(hM), _host(hN), _host(hK)))


def _host(a):
    """Host address of a contiguous int64 numpy array (kept alive by the caller)."""
    if a is None:
        return None
    return a.ctypes.data


def alp_tune(M, N, K, path=ALP_PATH_NATIVE, mode=ALP_TUNE_EXHAUSTIVE, raise_on_error=True):
    out = alp_config()
    tf = ctypes.c_double(0.0)
    st = lib().alp_tune(M, N, K, int(path), int(mode), ctypes.byref(out), ctypes.byref(tf))
    _check(st, "alp_tune", raise_on_error)
    return st, out, tf.value


def alp_get_device_error(stream=None):
    return int(lib().alp_get_device_error(_s(stream)))


def alp_config_valid(cfg, path=ALP_PATH_NATIVE) -> bool:
    c = cfg if isinstance(cfg, alp_config) else alp_config(*cfg)
    return bool(lib().alp_config_valid(ctypes.byref(c), int(path)))


def alp_config_smem_bytes(cfg) -> int:
    c = cfg if isinstance(cfg, alp_config) else alp_config(*cfg)
    return int(lib().alp_config_smem_bytes(ctypes.byref(c)))


def alp_config_threads(cfg) -> int:
    c = cfg if isinstance(cfg, alp_config) else alp_config(*cfg)
    return int(lib().alp_config_threads(ctypes.byref(c)))


def alp_config_count(path=ALP_PATH_NATIVE) -> int:
    return int(lib().alp_config_count(int(path)))


def alp_config_at(path, idx) -> alp_config:
    c = alp_config()
    st = lib().alp_config_at(int(path), int(idx), ctypes.byref(c))
    _check(st, "alp_config_at", True)
    return c


def alp_set_wait_timeout_ms(ms):
    return _check(lib().alp_set_wait_timeout_ms(float(ms)), "alp_set_wait_timeout_ms", True)


def alp_debug_inject_skip(kt):
    return _check(lib().alp_debug_inject_skip(int(kt)), "alp_debug_inject_skip", True)


def alp_probe_fp64_peak(kind=0, iters=20000, blocks_per_sm=2, threads=256, stream=None):
    """Measured FP64 TFLOP/s (kind 0: m16n8k4 DMMA chains, 1: DFMA chains, 2: m16n8k8
    DMMA chains, 3: m16n8k16 DMMA chains)."""
    out = ctypes.c_double(0.0)
    _check(lib().alp_probe_fp64_peak(int(kind), int(iters), int(blocks_per_sm), int(threads),
                                     ctypes.byref(out), _s(stream)), "alp_probe_fp64_peak", True)
    return out.value


def alp_emul_tail_split(tiles, nslices, kind, sms):
    """(n_full, [(t_lo, t_hi) per piece]) of the slice-product launch."""
    n_full, pieces = ctypes.c_int(0), ctypes.c_int(0)
    lo, hi = (_int * 8)(), (_int * 8)()
    _check(lib().alp_emul_tail_split(int(tiles), int(nslices), int(kind), int(sms),
                                     ctypes.byref(n_full),
                                     ctypes.byref(pieces), lo, hi), "alp_emul_tail_split", True)
    return n_full.value, [(lo[i], hi[i]) for i in range(pieces.value)]


def alp_batched_class_of(M, N) -> int:
    return int(lib().alp_batched_class_of(M, N))


def alp_batched_set_class_config(cls, bm, bn, bk):
    return _check(lib().alp_batched_set_class_config(int(cls), int(bm), int(bn), int(bk)),
                  "alp_batched_set_class_config", True)


def alp_batched_get_class_config(cls):
    bm, bn, bk = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().alp_batched_get_class_config(int(cls), ctypes.byref(bm), ctypes.byref(bn),
                                              ctypes.byref(bk)), "alp_batched_get_class_config",
           True)
    return bm.value, bn.value, bk.value


def alp_batched_graph_create(count, dM, dN, dK, dalpha, dA, dlda, dB, dldb, dbeta, dC, dldc,
                             hM, hN, hK, workspace, workspace_bytes):
    h = ctypes.c_void_p()
    st = lib().alp_batched_graph_create(count, _p(dM), _p(dN), _p(dK), _p(dalpha), _p(dA),
                                        _p(dlda), _p(dB), _p(dldb), _p(dbeta), _p(dC), _p(dldc),
                                        _host(hM), _host(hN), _host(hK), _p(workspace),
                                        int(workspace_bytes), ctypes.byref(h))
    _check(st, "alp_batched_graph_create", True)
    return h.value


def alp_batched_graph_launch(graph, stream=None):
    return _check(lib().alp_batched_graph_launch(graph, _s(stream)), "alp_batched_graph_launch",
                  True)


def alp_batched_graph_destroy(graph):
    return _check(lib().alp_batched_graph_destroy(graph), "alp_batched_graph_destroy", True)


def _cfg(c):
    return c if isinstance(c, alp_config) else alp_config(*c)


def alp_tune_time_config(M, N, K, path, cfg, use_proxy=True, runs=3):
    out = ctypes.c_double(0.0)
    c = _cfg(cfg)
    _check(lib().alp_tune_time_config(M, N, K, int(path), ctypes.byref(c), int(bool(use_proxy)),
                                      int(runs), ctypes.byref(out)), "alp_tune_time_config", True)
    return out.value


def alp_tune_set_cached(M, N, K, path, cfg):
    c = _cfg(cfg)
    return _check(lib().alp_tune_set_cached(M, N, K, int(path), ctypes.byref(c)),
                  "alp_tune_set_cached", True)


def alp_tune_clear_cache():
    return _check(lib().alp_tune_clear_cache(), "alp_tune_clear_cache", True)


def alp_mlp_param_count(C) -> int:
    return int(lib().alp_mlp_param_count(int(C)))


def alp_mlp_features(count, dM, dN, dK, dpath, mean, std, X, stream=None):
    return _check(lib().alp_mlp_features(count, _p(dM), _p(dN), _p(dK), _p(dpath), _p(mean),
                                         _p(std), _p(X), _s(stream)), "alp_mlp_features", True)


def alp_mlp_feature_stats(count, X, mean, std, stream=None):
    return _check(lib().alp_mlp_feature_stats(count, _p(X), _p(mean), _p(std), _s(stream)),
                  "alp_mlp_feature_stats", True)


def alp_mlp_forward(params, C, X, B, Y, cache, stream=None):
    return _check(lib().alp_mlp_forward(_p(params), int(C), _p(X), B, _p(Y), _p(cache),
                                        _s(stream)), "alp_mlp_forward", True)


def alp_mlp_backward(params, C, X, B, cache, Y, T, Mask, grads, work, loss, stream=None):
    return _check(lib().alp_mlp_backward(_p(params), int(C), _p(X), B, _p(cache), _p(Y), _p(T),
                                         _p(Mask), _p(grads), _p(work), _p(loss), _s(stream)),
                  "alp_mlp_backward", True)


def alp_mlp_adam(params, grads, m, v, n, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                 stream=None):
    return _check(lib().alp_mlp_adam(_p(params), _p(grads), _p(m), _p(v), n, int(step),
                                     float(lr), float(beta1), float(beta2), float(eps),
                                     _s(stream)), "alp_mlp_adam", True)


def alp_tune_load_model(host_params, C, host_mean, host_std):
    """host_* are contiguous float32 numpy arrays."""
    return _check(lib().alp_tune_load_model(host_params.ctypes.data, int(C),
                                            host_mean.ctypes.data, host_std.ctypes.data),
                  "alp_tune_load_model", True)


def alp_tune_unload_model():
    return _check(lib().alp_tune_unload_model(), "alp_tune_unload_model", True)


def alp_gemm_batched_varsize_noalloc(count, dM, dN, dK, dalpha, dA, dlda, dB, dldb, dbeta, dC,
                                     dldc, hM, hN, hK, stream=None, raise_on_error=True):
    """alp_gemm_batched_varsize without a workspace argument: the library's
    built-in 1 MiB scratch holds the work list (no device allocation)."""
    st = lib().alp_gemm_batched_varsize_noalloc(count, _p(dM), _p(dN), _p(dK), _p(dalpha),
                                                _p(dA), _p(dlda), _p(dB), _p(dldb), _p(dbeta),
                                                _p(dC), _p(dldc), _host(hM), _host(hN),
                                                _host(hK), _s(stream))
    return _check(st, "alp_gemm_batched_varsize_noalloc", raise_on_error)
