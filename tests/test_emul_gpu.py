"""Parity of the emulated FP64 GEMM (alp_gemm_f64_emul and its stages, through
the C-ABI) with the oracle's emulated-GEMM model: bit-exact exponents, digits
and results (every product and partial sum is exact and the single rounding
is fixed), plus its error against the long-double GEMM next to the native
path's."""
import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs

from .gpu_util import dev

pytestmark = pytest.mark.gpu


# slice kinds: name -> (alp_slice_kind value, digit bits b, trimmed last group)
KINDS = {"b7": (1, 7, False), "b8": (2, 8, False), "b8t": (3, 8, True)}


def model(orc, alpha, A, B, beta, C, s, kind="b7", rows=None):
    _, b, trim = KINDS[kind]
    return orc.emul_gemm(alpha, A, B, beta, C, s, b=b, trim=trim, rows=rows)


def run_emul(alp, A, B, C, alpha, beta, s, lda=None, ldc=None, raise_on_error=True, kind="b7"):
    import torch
    M, K = A.shape
    N = B.shape[1]
    dA, lda = dev(A, lda)
    dB, ldb = dev(B)
    dC, ldc = dev(C if C is not None else np.full((M, N), np.nan), ldc)
    k = KINDS[kind][0]
    ws = alp.alp_gemm_f64_emul_workspace(M, N, K, s, k)
    work = torch.empty(max(ws, 1), dtype=torch.uint8, device="cuda")
    st = alp.alp_gemm_f64_emul(M, N, K, alpha, dA, lda, dB, ldb, beta, dC, ldc, s, k, work, ws,
                               raise_on_error=raise_on_error)
    torch.cuda.synchronize()
    err = alp.alp_get_device_error()
    return dC.cpu().numpy()[:M, :N], st, err


def test_exponents_match_oracle(alp, orc):
    import torch
    A = inputs.scaled(3001, 0, (300, 200), phi=32)
    A[7] = 0.0
    A[11] = 0.0
    A[11, 5] = -2.0 ** -1060          # subnormal row maximum
    A[12, 3] = 2.0 ** 1000
    dA = torch.from_numpy(A).cuda()
    e = torch.empty(300, dtype=torch.int32, device="cuda")
    alp.alp_emul_exponents(300, 200, dA, 200, 0, e)
    ref, bad = orc.row_exponents(A)
    assert not bad and np.array_equal(e.cpu().numpy(), ref)
    B = inputs.scaled(3002, 0, (700, 130), phi=32)     # K = 700 spans several column chunks
    B[:, 4] = 0.0
    B[:, 9] = 0.0
    B[650, 9] = 2.0 ** -1070
    dB = torch.from_numpy(B).cuda()
    f = torch.empty(130, dtype=torch.int32, device="cuda")
    alp.alp_emul_exponents(130, 700, dB, 130, 1, f)
    torch.cuda.synchronize()
    ref, bad = orc.col_exponents(B)
    assert not bad and np.array_equal(f.cpu().numpy(), ref)
    assert alp.alp_get_device_error() == alp.ALP_OK


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("off,ld_pad,R,K", [(0, 0, 37, 1000), (1, 3, 37, 1001), (3, 0, 5, 7),
                                            (0, 1, 9, 2), (2, 2, 300, 515)])
def test_exponents_vector_and_ragged_paths(alp, orc, dtype, off, ld_pad, R, K):
    """Row and column scans on views whose base is off elements past a 16-byte
    boundary and whose leading dimension is padded: the aligned vector body,
    the unaligned head, the ragged tail and the element-by-element column
    path; one Inf and one NaN are reported and do not affect other rows."""
    import torch
    X = inputs.scaled(3003 + off + K, 0, (R, K), phi=40)
    X[1] = 0.0
    X[2, K - 1] = 2.0 ** 600 if dtype == "f64" else 2.0 ** 100
    X[3, 0] = -(2.0 ** -1060) if dtype == "f64" else -(2.0 ** -140)
    X[3, 1:] = 0.0
    npdt = np.float64 if dtype == "f64" else np.float32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Xc = X.astype(npdt)
    ld = K + ld_pad
    buf = torch.zeros(off + R * ld + 8, dtype=tdt, device="cuda")
    view = buf[off:off + R * ld].view(R, ld)
    view[:, :K] = torch.from_numpy(Xc)
    scan = alp.alp_emul_exponents if dtype == "f64" else alp.alp_emul_exponents_f32
    e = torch.empty(R, dtype=torch.int32, device="cuda")
    scan(R, K, view, ld, 0, e)
    torch.cuda.synchronize()
    ref, _ = orc.row_exponents(Xc.astype(np.float64))
    assert np.array_equal(e.cpu().numpy(), ref)
    # the same values stored K x R (columns), leading dimension ld2
    XT = np.ascontiguousarray(Xc.T)
    ld2 = R + ld_pad
    buf2 = torch.zeros(off + K * ld2 + 8, dtype=tdt, device="cuda")
    view2 = buf2[off:off + K * ld2].view(K, ld2)
    view2[:, :R] = torch.from_numpy(XT)
    f = torch.empty(R, dtype=torch.int32, device="cuda")
    scan(R, K, view2, ld2, 1, f)
    torch.cuda.synchronize()
    assert np.array_equal(f.cpu().numpy(), ref)
    assert alp.alp_get_device_error() == alp.ALP_OK
    view[4, K // 2] = float("inf")
    view2[K // 2, 4] = float("nan")
    scan(R, K, view, ld, 0, e)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_ERR_UNSUPPORTED
    got = e.cpu().numpy()
    assert np.array_equal(np.delete(got, 4), np.delete(ref, 4))
    scan(R, K, view2, ld2, 1, f)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_ERR_UNSUPPORTED
    assert np.array_equal(np.delete(f.cpu().numpy(), 4), np.delete(ref, 4))


@pytest.mark.parametrize("phi", [0, 8, 32])
@pytest.mark.parametrize("s,kind", [(8, "b7"), (7, "b8"), (3, "b8"), (7, "b8t")])
def test_split_matches_oracle(alp, orc, phi, s, kind):
    import torch
    R, K = 70, 150
    kpad = 192
    X = inputs.scaled(3010 + phi, 0, (R, K), phi)
    X[0, :8] = [0.5, -0.5, 0.75, 1.0 / 256, 3.0 / 512, -2.0 ** -9, 2.0 ** -60, 0.0]  # ties, tiny
    X[1] = 0.0
    X[2, :4] = [1.0 - 2.0 ** -53, -(1.0 - 2.0 ** -53), 0.5 + 2.0 ** -10, 1.0 / 512]
    e, _ = orc.row_exponents(X)
    k, b, _ = KINDS[kind]
    ref, _ = orc.split(X, e, s, b)
    assert np.abs(ref[0]).max() <= 2 ** b and np.abs(ref[1:]).max() <= 2 ** (b - 1)
    dX = torch.from_numpy(X).cuda()
    de = torch.from_numpy(e).cuda()
    out = torch.full((s, R, kpad), 7.0, dtype=torch.bfloat16, device="cuda")
    alp.alp_emul_split(R, K, dX, K, 0, de, s, k, out, kpad)
    got = out.float().cpu().numpy()
    assert np.array_equal(got[:, :, :K], ref.astype(np.float32))
    assert np.all(got[:, :, K:] == 0.0)
    # transposed input: a K x R row-major matrix whose columns are split
    XT = np.ascontiguousarray(X.T)
    out2 = torch.full((s, R, kpad), 7.0, dtype=torch.bfloat16, device="cuda")
    alp.alp_emul_split(R, K, torch.from_numpy(XT).cuda(), R, 1, de, s, k, out2, kpad)
    got2 = out2.float().cpu().numpy()
    assert np.array_equal(got2[:, :, :K], ref.astype(np.float32))
    assert np.all(got2[:, :, K:] == 0.0)


SHAPES = [(128, 256, 64), (200, 300, 130), (1, 1, 1), (257, 513, 1000), (64, 40, 2049)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("s,phi", [(3, 0), (8, 0), (8, 32), (5, 8)])
def test_emul_bit_exact_vs_model(alp, orc, shape, s, phi):
    M, N, K = shape
    A, B, C = inputs.gemm_operands(3100 + M + N + K + s + phi, M, N, K, kind="scaled", phi=phi)
    got, st, err = run_emul(alp, A, B, C, 1.5, 0.5, s)
    assert st == alp.ALP_OK and err == alp.ALP_OK
    ref, rc = orc.emul_gemm(1.5, A, B, 0.5, C, s)
    assert rc == 0
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["b8", "b8t"])
@pytest.mark.parametrize("s,phi", [(3, 0), (6, 0), (7, 0), (7, 32), (5, 8)])
def test_emul_8bit_digits_bit_exact_vs_model(alp, orc, shape, kind, s, phi):
    """8-bit digits (ALP_SLICE_BF16_B8) and the trimmed last group
    (ALP_SLICE_BF16_B8_TRIM): the same model with b = 8."""
    M, N, K = shape
    A, B, C = inputs.gemm_operands(3700 + M + N + K + s + phi, M, N, K, kind="scaled", phi=phi)
    got, st, err = run_emul(alp, A, B, C, 1.5, 0.5, s, kind=kind)
    assert st == alp.ALP_OK and err == alp.ALP_OK
    ref, rc = model(orc, 1.5, A, B, 0.5, C, s, kind)
    assert rc == 0
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("bm,cluster,group", [(128, 1, 1), (128, 1, 4), (128, 1, 8), (128, 1, 32),
                                              (256, 2, 1), (256, 2, 8), (256, 2, 32)])
def test_emul_every_config_bit_exact(alp, orc, bm, cluster, group):
    """Each emulated config (one block per tile, CTA pairs sharing each MMA;
    raster group), forced through the tuned cache, on a shape with an odd
    number of tile-rows and ragged edges."""
    M, N, K = 3 * 128 + 5, 2 * 256 + 9, 700
    cfg = (bm, 256, 64, cluster, 0, group)
    assert alp.alp_config_valid(cfg, alp.ALP_PATH_EMUL)
    A, B, C = inputs.gemm_operands(3600 + bm + cluster * 100 + group, M, N, K, kind="scaled",
                                   phi=8)
    alp.alp_tune_set_cached(M, N, K, alp.ALP_PATH_EMUL, cfg)
    try:
        runs = (("b7", 8), ("b8", 7), ("b8t", 7))
        got = [run_emul(alp, A, B, C, 1.5, 0.5, s, kind=kind) for kind, s in runs]
    finally:
        alp.alp_tune_clear_cache()
    for (kind, s), (res, st, err) in zip(runs, got):
        assert err == alp.ALP_OK
        ref, _ = model(orc, 1.5, A, B, 0.5, C, s, kind)
        assert np.array_equal(res, ref), kind


# rows of a 130-row result on both sides of the 128-row tile edge
EDGE_ROWS = np.array([0, 1, 63, 127, 128, 129])


@pytest.mark.parametrize("K", [63, 64, 65, 1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097,
                               8193])
def test_emul_chunk_boundaries(alp, orc, K):
    """K around the 7-bit drain chunks (1024, 2048, 4096) and the 64-wide
    k-blocks; the result on rows across the tile edge, every column."""
    M, N = 130, 260
    A, B, _ = inputs.gemm_operands(3200 + K, M, N, K, kind="scaled", phi=4, with_c=False)
    got, st, err = run_emul(alp, A, B, None, 1.0, 0.0, 8)
    assert err == alp.ALP_OK
    ref, _ = orc.emul_gemm(1.0, A, B, 0.0, None, 8, rows=EDGE_ROWS)
    assert np.array_equal(got[EDGE_ROWS], ref)


@pytest.mark.parametrize("K", [255, 256, 257, 511, 512, 513, 1023, 1024, 1025, 2000])
@pytest.mark.parametrize("kind", ["b8", "b8t"])
def test_emul_8bit_chunk_boundaries(alp, orc, K, kind):
    """8-bit digits drain every 256, 512 or 1024 k: K around those chunks."""
    M, N = 130, 260
    A, B, _ = inputs.gemm_operands(3800 + K, M, N, K, kind="scaled", phi=4, with_c=False)
    got, st, err = run_emul(alp, A, B, None, 1.0, 0.0, 7, kind=kind)
    assert err == alp.ALP_OK
    ref, _ = model(orc, 1.0, A, B, 0.0, None, 7, kind, rows=EDGE_ROWS)
    assert np.array_equal(got[EDGE_ROWS], ref)


@pytest.mark.parametrize("kind,s", [("b7", 8), ("b8", 7), ("b8t", 7)])
def test_emul_partial_sums_at_the_chunk_bound(alp, orc, kind, s):
    """Entries whose first three digits are 2^b, -2^(b-1), 2^(b-1) (a tie at
    each of the first two steps): every product of pairs among the first three
    digits is at its bound, and with equal signs along k each chunk's f32
    partial sum reaches exactly +-2^24, the largest the chunking allows.  Rows
    of A flip sign and carry a second pattern, so both signs of the bound occur."""
    _, b, _ = KINDS[kind]
    x = (2.0 ** b - 0.5 + 2.0 ** (-b - 1)) / 2.0 ** b
    d, _ = orc.split(np.array([[x]]), np.array([0], dtype=np.int32), 4, b)
    assert list(d[:, 0, 0]) == [2 ** b, -2 ** (b - 1), 2 ** (b - 1), 0]
    M, N = 130, 260
    K = 2 ** (26 - 2 * b)                       # one chunk of the pairs without a first digit
    A = np.full((M, K), x)
    A[1::2] *= -1
    A[2::3, ::2] = 0.5                          # second pattern: digits (2^(b-1), 0, ...)
    B = np.full((K, N), x)
    B[:, 1::4] *= -1
    got, st, err = run_emul(alp, A, B, None, 1.0, 0.0, s, kind=kind)
    assert err == alp.ALP_OK
    rows = np.array([0, 1, 2, 3, 4, 5, 63, 127, 128, 129])
    ref, _ = model(orc, 1.0, A, B, 0.0, None, s, kind, rows=rows)
    assert np.array_equal(got[rows], ref)


@pytest.mark.parametrize("kind,s", [("b7", 8), ("b8", 7), ("b8t", 7)])
def test_emul_largest_k(alp, orc, kind, s):
    """K at the int32 group-sum limit (32768 for 7-bit digits, 14336 for
    8-bit); row 0 has its leading digit at the bound 2^b with signs matching
    B's, so its first group sum S^2 is K * 2^(2b), the largest one; one past
    the limit is refused."""
    M, N = 130, 40
    b = KINDS[kind][1]
    K = 32768 if b == 7 else 14336
    A = np.full((M, K), 1.0 - 2.0 ** -53)
    A[:, 1::2] *= -1
    A[1:] = inputs.scaled(3900 + b, 0, (M - 1, K), 0)
    B = np.full((K, N), 1.0 - 2.0 ** -53)
    B[1::2, :] *= -1
    got, st, err = run_emul(alp, A, B, None, 1.0, 0.0, s, kind=kind)
    assert st == alp.ALP_OK and err == alp.ALP_OK
    rows = np.array([0, 1, 77, M - 1])
    ref, _ = model(orc, 1.0, A, B, 0.0, None, s, kind, rows=rows)
    assert np.array_equal(got[rows], ref)
    _, st, _ = run_emul(alp, np.zeros((8, K + 1)), np.zeros((K + 1, 8)), None, 1.0, 0.0, s,
                        kind=kind, raise_on_error=False)
    assert st == alp.ALP_ERR_UNSUPPORTED


@pytest.mark.parametrize("kind", ["b7", "b8", "b8t"])
def test_emul_worst_case_digits_exact_b(alp, orc, kind):
    """Near-maximal alternating entries for either digit width: every digit at
    or next to its bound, partial sums as large as the chunking allows."""
    M, N, K = 128, 256, 1024
    A = np.full((M, K), 1.0 - 2.0 ** -53)
    A[:, 1::2] *= -1
    B = np.full((K, N), 1.0 - 2.0 ** -53)
    B[1::2, :] *= -1
    s = 8 if kind == "b7" else 7
    got, st, err = run_emul(alp, A, B, None, 1.0, 0.0, s, kind=kind)
    ref, _ = model(orc, 1.0, A, B, 0.0, None, s, kind)
    assert np.array_equal(got, ref)


def test_emul_worst_case_digits_exact(alp, orc):
    """Entries whose digits are all at their bounds (|d_1| = 128 and |d_p| = 64
    would need a tie, so near-maximal values): the largest partial sums the
    chunking allows, still exact."""
    M, N, K = 128, 256, 1024
    A = np.full((M, K), 1.0 - 2.0 ** -53)
    A[:, 1::2] *= -1
    B = np.full((K, N), 1.0 - 2.0 ** -53)
    B[1::2, :] *= -1
    got, st, err = run_emul(alp, A, B, None, 1.0, 0.0, 8)
    ref, _ = orc.emul_gemm(1.0, A, B, 0.0, None, 8)
    assert np.array_equal(got, ref)


def test_emul_extreme_exponents(alp, orc):
    """Rows and columns scaled far apart: results that underflow to
    subnormals (one rounding) or overflow to infinity, bit-exact."""
    M, N, K = 70, 90, 50
    A, B, C = inputs.gemm_operands(3500, M, N, K)
    A[:20] *= 2.0 ** -1000
    B[:, :30] *= 2.0 ** -60
    A[20:40] *= 2.0 ** 900
    B[:, 30:60] *= 2.0 ** 200
    got, st, err = run_emul(alp, A, B, C, 1.0, 0.0, 8)
    ref, _ = orc.emul_gemm(1.0, A, B, 0.0, None, 8)
    assert np.array_equal(got, ref)
    assert np.isinf(got).any() and (np.abs(got[:20, :30]) < 2.0 ** -1022).all()


def test_emul_integer_inputs_exact(alp, orc):
    M = N = K = 512
    A, B, _ = inputs.gemm_operands(inputs.workload_seed("dgemm_512"), M, N, K, kind="int",
                                   with_c=False)
    got, _, _ = run_emul(alp, A, B, None, 1.0, 0.0, 3)
    assert np.array_equal(got, orc.gemm(1.0, A, B, 0.0))


def test_emul_alpha_beta_and_padding(alp, orc):
    M, N, K = 100, 70, 90
    A, B, C = inputs.gemm_operands(3300, M, N, K)
    got, _, _ = run_emul(alp, np.full_like(A, np.nan), np.full_like(B, np.nan), C, 0.0, 0.5, 6)
    assert np.array_equal(got, 0.5 * C)
    got, _, _ = run_emul(alp, A, B, np.full_like(C, np.nan), 1.0, 0.0, 6)
    ref, _ = orc.emul_gemm(1.0, A, B, 0.0, None, 6)
    assert np.array_equal(got, ref)
    got, _, _ = run_emul(alp, A, B, C, -2.0, 0.25, 6, lda=K + 3, ldc=N + 5)
    ref, _ = orc.emul_gemm(-2.0, A, B, 0.25, C, 6)
    assert np.array_equal(got, ref)


def test_emul_inf_nan_and_unsupported(alp, orc):
    M, N, K = 64, 64, 64
    A, B, C = inputs.gemm_operands(3400, M, N, K)
    A[3, 4] = np.inf
    _, st, err = run_emul(alp, A, B, C, 1.0, 0.0, 8)
    assert st == alp.ALP_OK and err == alp.ALP_ERR_UNSUPPORTED
    B[5, 6] = np.nan
    A[3, 4] = 1.0
    _, st, err = run_emul(alp, A, B, C, 1.0, 0.0, 8)
    assert err == alp.ALP_ERR_UNSUPPORTED
    assert alp.alp_get_device_error() == alp.ALP_OK      # read-and-clear
    assert alp.alp_gemm_f64_emul(4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, 8, alp.ALP_SLICE_INT8,
                                 None, 0, stream=0, raise_on_error=False) == alp.ALP_ERR_UNSUPPORTED
    assert alp.alp_gemm_f64_emul(4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, 9, alp.ALP_SLICE_BF16,
                                 None, 0, stream=0, raise_on_error=False) == alp.ALP_ERR_INVALID_ARG
    assert alp.alp_gemm_f64_emul(4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, 8, alp.ALP_SLICE_BF16,
                                 None, 0, stream=0, raise_on_error=False) == alp.ALP_ERR_WORKSPACE
    assert alp.alp_gemm_f64_emul(4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, 8, alp.ALP_SLICE_BF16_B8,
                                 None, 0, stream=0, raise_on_error=False) == alp.ALP_ERR_INVALID_ARG
    assert alp.alp_gemm_f64_emul(4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, 7, 5, None, 0, stream=0,
                                 raise_on_error=False) == alp.ALP_ERR_INVALID_ARG   # no kind 5
    assert alp.alp_gemm_f64_emul(4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, 8, alp.ALP_SLICE_BF16_B8_TRIM,
                                 None, 0, stream=0, raise_on_error=False) == alp.ALP_ERR_INVALID_ARG
    assert alp.alp_gemm_f64_emul_workspace(64, 64, 64, 8, alp.ALP_SLICE_BF16_B8) == 0
    assert alp.alp_gemm_f64_emul_workspace(64, 64, 64, 7, alp.ALP_SLICE_BF16_B8) > 0
    assert alp.alp_gemm_f64_emul_workspace(64, 64, 64, 8, alp.ALP_SLICE_BF16_B8_TRIM) == 0
    assert alp.alp_gemm_f64_emul_workspace(64, 64, 64, 7, alp.ALP_SLICE_BF16_B8_TRIM) > 0
    assert alp.alp_gemm_f64_emul_workspace(64, 64, 64, 7, 5) == 0


def componentwise_ratio(got, ref, absAB, alpha, beta, C):
    den = abs(alpha) * absAB + (np.abs(beta * C) if beta != 0 else 0.0)
    return float(np.max(np.abs(got - ref) / np.maximum(den, 1e-300)))


def test_emul_error_no_worse_than_native(alp, orc):
    """phi = 0, s = 8: the emulated result's largest componentwise error,
    relative to |alpha||A||B| + |beta C|, is at most the native kernel's."""
    from .test_native_gpu import run_gemm
    M = N = K = 1024
    A, B, C = inputs.gemm_operands(inputs.workload_seed("emul_8192"), M, N, K, kind="scaled",
                                   phi=0)
    rows = np.arange(0, M, 16)
    ref = orc.gemm(1.5, A, B, 0.5, C, rows=rows)
    absAB = orc.absgemm(A, B, rows=rows)
    emul, _, _ = run_emul(alp, A, B, C, 1.5, 0.5, 8)
    nat, _ = run_gemm(alp, A, B, C, 1.5, 0.5)
    r_emul = componentwise_ratio(emul[rows], ref, absAB, 1.5, 0.5, C[rows])
    r_nat = componentwise_ratio(nat[rows], ref, absAB, 1.5, 0.5, C[rows])
    assert r_emul <= r_nat, (r_emul, r_nat)
    # and within the acceptance bound of the native path
    bound = orc.error_bound(1.5, absAB, 0.5, C[rows], K)
    assert np.all(np.abs(emul[rows] - ref) <= bound)


def test_emul_full_size_sampled_rows(alp, orc):
    """M = N = K = 8192, phi = 8, s = 8, in the bench's launch configuration:
    sampled rows bit-exact against the model."""
    M = N = K = 8192
    A, B, _ = inputs.gemm_operands(inputs.workload_seed("emul_8192"), M, N, K, kind="scaled",
                                   phi=8, with_c=False)
    rows = np.array([0, 4097, 8191])
    for s, kind in ((8, "b7"), (7, "b7"), (6, "b8"), (7, "b8t")):
        got, st, err = run_emul(alp, A, B, None, 1.0, 0.0, s, kind=kind)
        assert err == alp.ALP_OK
        ref, _ = model(orc, 1.0, A, B, 0.0, None, s, kind, rows=rows)
        assert np.array_equal(got[rows], ref), (s, kind)


@pytest.mark.parametrize("kind,s", [("b7", 8), ("b7", 3), ("b8", 7), ("b8", 5)])
def test_recombine_rounding(alp, kind, s):
    """alp_emul_recombine on crafted group sums: X = sum_t S^t 2^(b(s+1-t))
    whose tails are exact ties, just below or above a tie, sticky bits far
    below, negative, zero, and scalings into the subnormal and overflow
    ranges; each result must be Python's correctly rounded float(X) scaled by
    ldexp (one more rounding when subnormal), i.e. the definition."""
    import math
    import random

    import torch
    k, b, _ = KINDS[kind]
    rnd = random.Random(17 + s + b)
    vals = []
    for _ in range(600):
        nbits = rnd.randrange(1, 31 + b * (s - 1))
        X = rnd.getrandbits(nbits) | (1 << (nbits - 1))
        form = rnd.randrange(5)
        if nbits > 54 and form < 4:
            # r: the bit just below the 53 kept; forms: exact tie, just below, just
            # above, and a lone sticky bit somewhere below
            r = nbits - 54 if form < 3 else rnd.randrange(0, nbits - 54)
            X = (X >> (r + 1)) << (r + 1)
            X += [1 << r, (1 << r) - 1, (1 << r) + 1, 1 << r][form]
        vals.append(-X if rnd.random() < 0.5 else X)
    vals += [v for v in (0, 1, -1, 2 ** 53 + 1, 2 ** 54 + 2, -(2 ** 54 + 6))
             if abs(v) < 2 ** (30 + b * (s - 1))]
    N = len(vals)
    ldg = (N + 255) // 256 * 256
    rows = 3
    G = np.zeros((s, rows, ldg), dtype=np.int32)
    for j, X in enumerate(vals):
        # base-2^b digits, the top one signed and unbounded within int32
        digits = []
        rest = X
        for _ in range(s - 1):
            digits.append(rest & ((1 << b) - 1))
            rest >>= b
        assert -2 ** 31 <= rest < 2 ** 31
        col = [rest] + digits[::-1]
        for row in range(rows):
            G[:, row, j] = col
    e = np.array([0, -1000, 200], dtype=np.int32)       # rows 1, 2: subnormal, overflow
    f = np.array([rnd.choice([0, 5, -3, 900, -60]) for _ in range(N)], dtype=np.int32)
    dG, de, df = (torch.from_numpy(x).cuda() for x in (G, e, f))
    dC = torch.full((rows, N), np.nan, dtype=torch.float64, device="cuda")
    alp.alp_emul_recombine(rows, N, s, k, dG, ldg, de, df, 1.0, 0.0, dC, N)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    for row in range(rows):
        for j, X in enumerate(vals):
            E = int(e[row]) + int(f[j]) - (s + 1) * b
            try:
                want = math.ldexp(float(X), E)
            except OverflowError:
                want = math.copysign(math.inf, X)
            assert got[row, j] == want or (want == 0 and got[row, j] == 0), (row, j, X, E)


@pytest.mark.parametrize("ta,tb", [(0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("kind,s", [("b7", 8), ("b8t", 7)])
def test_emul_transposed_operands_bit_exact(alp, orc, ta, tb, kind, s):
    """alp_gemm_f64_emul_ex with op(A) = A^T and/or op(B) = B^T, padded leading
    dimensions: the oracle's result on the transposed matrices."""
    import torch
    M, N, K = 3 * 128 + 5, 2 * 256 + 9, 700
    A, B, C = inputs.gemm_operands(4400 + 2 * ta + tb, M, N, K, kind="scaled", phi=8)
    As = np.ascontiguousarray(A.T) if ta else A            # stored K x M or M x K
    Bs = np.ascontiguousarray(B.T) if tb else B            # stored N x K or K x N
    lda, ldb = As.shape[1] + 3, Bs.shape[1] + 5
    dA = torch.full((As.shape[0], lda), float("nan"), dtype=torch.float64, device="cuda")
    dA[:, :As.shape[1]] = torch.from_numpy(As)
    dB = torch.full((Bs.shape[0], ldb), float("nan"), dtype=torch.float64, device="cuda")
    dB[:, :Bs.shape[1]] = torch.from_numpy(Bs)
    dC = torch.from_numpy(C).cuda()
    k = KINDS[kind][0]
    ws = alp.alp_gemm_f64_emul_workspace(M, N, K, s, k)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    alp.alp_gemm_f64_emul_ex(ta, tb, M, N, K, 1.5, dA, lda, dB, ldb, 0.5, dC, N, s, k, work, ws)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    ref, _ = model(orc, 1.5, A, B, 0.5, C, s, kind)
    assert np.array_equal(dC.cpu().numpy(), ref)
    bad = alp.alp_gemm_f64_emul_ex(ta, tb, M, N, K, 1.5, dA, (M if ta else K) - 1, dB, ldb, 0.5,
                                   dC, N, s, k, work, ws, raise_on_error=False)
    assert bad == alp.ALP_ERR_INVALID_ARG
    assert alp.alp_gemm_f64_emul_ex(2, 0, M, N, K, 1.5, dA, lda, dB, ldb, 0.5, dC, N, s, k, work,
                                    ws, raise_on_error=False) == alp.ALP_ERR_INVALID_ARG


def test_emul_host_resident_operands(alp, orc):
    """On a device that reads host memory through the host's page tables
    (alp_host_access), A, B and C may live in ordinary (pageable) host memory:
    the scans and splits read them there, the recombination writes C there.
    Same bits as with device-resident operands; skipped elsewhere."""
    import torch
    pageable, _ = alp.alp_host_access()
    if not pageable:
        pytest.skip("this device does not access pageable host memory")
    M, N, K = 3 * 128 + 5, 2 * 256 + 9, 700
    A, B, C = inputs.gemm_operands(4600, M, N, K, kind="scaled", phi=8)
    A, B = np.ascontiguousarray(A), np.ascontiguousarray(B)
    hC = np.ascontiguousarray(C.copy())
    k = alp.ALP_SLICE_BF16_B8_TRIM
    ws = alp.alp_gemm_f64_emul_workspace(M, N, K, 7, k)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    alp.alp_gemm_f64_emul(M, N, K, 1.5, A.ctypes.data, K, B.ctypes.data, N, 0.5, hC.ctypes.data,
                          N, 7, k, work, ws)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    ref, _ = orc.emul_gemm(1.5, A, B, 0.5, C, 7, b=8, trim=True)
    assert np.array_equal(hC, ref)
