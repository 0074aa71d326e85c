"""Column-major (BLAS) entry points through the C-ABI: matrices stored column
by column with padded leading dimensions and every trans combination.  The
emulated calls must reproduce the oracle's results on op(A) op(B) bit for bit
(the same scaling exponents and the same exact integer products per element);
the native call must meet the FP64 error bound against the long-double
oracle.  Padding of C stays untouched."""
import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs

from .gpu_util import assert_within_bound

pytestmark = pytest.mark.gpu

CRT_MODULI = [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193]


def crt_k(K, n):
    Mn = 1
    for m in CRT_MODULI[:n]:
        Mn *= m
    return next(k for k in range(60, 0, -1) if K * 2 ** (2 * k + 1) <= Mn - (Mn >> 18))


def colmajor(X, pad, dtype):
    """Device buffer holding X (r x c) column-major with leading dimension
    r + pad (the row-major storage of X^T), padding NaN."""
    import torch
    r, c = X.shape
    buf = np.full((c, r + pad), np.nan, dtype=dtype)
    buf[:, :r] = X.T
    return torch.from_numpy(buf).cuda(), r + pad


def from_colmajor(t, r, c):
    buf = t.cpu().numpy()
    return np.ascontiguousarray(buf[:, :r].T), buf[:, r:]


TRANS = [(0, 0), (0, 1), (1, 0), (1, 1)]


def operands(seed, M, N, K, ta, tb, dtype):
    A, B, C = inputs.gemm_operands(seed, M, N, K, kind="scaled", phi=4)
    A, B, C = (x.astype(dtype) for x in (A, B, C))
    # the stored matrices: op(A) = A_s or A_s^T
    A_s = np.ascontiguousarray(A.T) if ta else A
    B_s = np.ascontiguousarray(B.T) if tb else B
    return A, B, C, A_s, B_s


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("kind,s", [(4, 15), (3, 7)])
def test_emul_f64_colmajor_bit_exact(alp, orc, ta, tb, kind, s):
    import torch
    M, N, K = 257, 300, 333
    A, B, C, A_s, B_s = operands(6100 + 2 * ta + tb, M, N, K, ta, tb, np.float64)
    dA, lda = colmajor(A_s, 3, np.float64)
    dB, ldb = colmajor(B_s, 5, np.float64)
    dC, ldc = colmajor(C, 7, np.float64)
    ws = alp.alp_gemm_f64_emul_cm_workspace(M, N, K, s, kind)
    assert ws == alp.alp_gemm_f64_emul_workspace(N, M, K, s, kind) > 0
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    alp.alp_gemm_f64_emul_cm(ta, tb, M, N, K, 1.5, dA, lda, dB, ldb, 0.5, dC, ldc, s, kind, work, ws)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    got, pad = from_colmajor(dC, M, N)
    if kind == 4:
        ref, _ = orc.crt_gemm(1.5, A, B, 0.5, C, crt_k(K, s))
    else:
        ref, _ = orc.emul_gemm(1.5, A, B, 0.5, C, s, b=8, trim=True)
    assert np.array_equal(got, ref)
    assert np.all(np.isnan(pad))
    # a leading dimension below the stored rows is rejected before any launch
    assert alp.alp_gemm_f64_emul_cm(ta, tb, M, N, K, 1.5, dA, (K if ta else M) - 1, dB, ldb, 0.5,
                                    dC, ldc, s, kind, work, ws,
                                    raise_on_error=False) == alp.ALP_ERR_INVALID_ARG


@pytest.mark.parametrize("ta,tb", TRANS)
def test_emul_f32_colmajor_bit_exact(alp, orc, ta, tb):
    import torch
    M, N, K = 200, 130, 260
    A, B, C, A_s, B_s = operands(6200 + 2 * ta + tb, M, N, K, ta, tb, np.float32)
    dA, lda = colmajor(A_s, 1, np.float32)
    dB, ldb = colmajor(B_s, 2, np.float32)
    dC, ldc = colmajor(C, 3, np.float32)
    kind = alp.ALP_SLICE_BF16_B8
    ws = alp.alp_gemm_f32_emul_cm_workspace(M, N, K, 3, kind)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    alp.alp_gemm_f32_emul_cm(ta, tb, M, N, K, 1.5, dA, lda, dB, ldb, 0.5, dC, ldc, 3, kind, work,
                             ws)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    got, pad = from_colmajor(dC, M, N)
    ref, _ = orc.emul_gemm_f32(1.5, A, B, 0.5, C, 3, b=8)
    assert np.array_equal(got, ref)
    assert np.all(np.isnan(pad))


@pytest.mark.parametrize("ta,tb", TRANS)
def test_native_colmajor_within_bound(alp, orc, ta, tb):
    import torch
    M, N, K = 300, 257, 190
    A, B, C, A_s, B_s = operands(6300 + 2 * ta + tb, M, N, K, ta, tb, np.float64)
    dA, lda = colmajor(A_s, 3, np.float64)
    dB, ldb = colmajor(B_s, 1, np.float64)
    dC, ldc = colmajor(C, 2, np.float64)
    ws = alp.alp_gemm_f64_cm_workspace(ta, tb, M, N, K)
    assert ws == alp.alp_gemm_f64_ex_workspace(tb, ta, N, M, K)
    work = torch.empty(max(ws, 1), dtype=torch.uint8, device="cuda")
    alp.alp_gemm_f64_cm(ta, tb, M, N, K, 1.5, dA, lda, dB, ldb, 0.5, dC, ldc, None, work, ws)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    got, pad = from_colmajor(dC, M, N)
    ref = orc.gemm(1.5, A, B, 0.5, C)
    assert_within_bound(got, ref, orc.absgemm(A, B), 1.5, 0.5, C, K)
    assert np.all(np.isnan(pad))
