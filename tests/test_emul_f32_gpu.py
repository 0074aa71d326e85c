"""Parity of the emulated FP32 GEMM (alp_gemm_f32_emul and its stages, through
the C-ABI) with the oracle's FP32 emulated-GEMM model: bit-exact digits and
results, plus its error against the long-double GEMM next to the FP32 GEMM
of the vendor library (a comparison only, not a path of this library)."""
import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs

pytestmark = pytest.mark.gpu

# slice kinds: name -> (alp_slice_kind value, digit bits b, trimmed last group)
KINDS = {"b7": (1, 7, False), "b8": (2, 8, False), "b8t": (3, 8, True)}


def f32(*xs):
    return tuple(np.ascontiguousarray(x, dtype=np.float32) for x in xs)


def run_emul_f32(alp, A, B, C, alpha, beta, s, kind="b8", lda=None, ldc=None,
                 raise_on_error=True):
    import torch
    M, K = A.shape
    N = B.shape[1]
    lda = lda or K
    ldc = ldc or N
    dA = torch.full((M, lda), float("nan"), dtype=torch.float32, device="cuda")
    dA[:, :K] = torch.from_numpy(A)
    dB = torch.from_numpy(B).cuda()
    dC = torch.full((M, ldc), float("nan"), dtype=torch.float32, device="cuda")
    if C is not None:
        dC[:, :N] = torch.from_numpy(C)
    k = KINDS[kind][0]
    ws = alp.alp_gemm_f32_emul_workspace(M, N, K, s, k)
    work = torch.empty(max(ws, 1), dtype=torch.uint8, device="cuda")
    st = alp.alp_gemm_f32_emul(M, N, K, alpha, dA, lda, dB, N, beta, dC, ldc, s, k, work, ws,
                               raise_on_error=raise_on_error)
    torch.cuda.synchronize()
    err = alp.alp_get_device_error()
    return dC.cpu().numpy()[:, :N], st, err, dC.cpu().numpy()


def model(orc, alpha, A, B, beta, C, s, kind, rows=None):
    _, b, trim = KINDS[kind]
    return orc.emul_gemm_f32(alpha, A, B, beta, C, s, b=b, trim=trim, rows=rows)


SHAPES = [(128, 256, 64), (200, 300, 130), (1, 1, 1), (257, 513, 1000), (64, 40, 2049)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("s,kind,phi", [(3, "b8", 0), (2, "b8", 0), (4, "b8", 8), (3, "b8t", 4),
                                        (4, "b7", 0), (3, "b7", 16)])
def test_emul_f32_bit_exact_vs_model(alp, orc, shape, s, kind, phi):
    M, N, K = shape
    A, B, C = inputs.gemm_operands(4100 + M + N + K + s + phi, M, N, K, kind="scaled", phi=phi)
    A, B, C = f32(A, B, C)
    got, st, err, _ = run_emul_f32(alp, A, B, C, 1.5, 0.5, s, kind)
    assert st == alp.ALP_OK and err == alp.ALP_OK
    ref, rc = model(orc, 1.5, A, B, 0.5, C, s, kind)
    assert rc == 0
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("s,kind", [(3, "b8"), (4, "b7")])
def test_split_f32_matches_oracle(alp, orc, s, kind):
    """Digits of float operands (rows and transposed columns) equal the
    oracle's digits of the same values as doubles."""
    import torch
    k, b, _ = KINDS[kind]
    R, K, kpad = 70, 150, 192
    X = f32(inputs.scaled(4200, 0, (R, K), 8))[0]
    X[0, :4] = [0.5, -0.75, 2.0 ** -30, 0.0]
    X[1] = 0.0
    X64 = X.astype(np.float64)
    e, _ = orc.row_exponents(X64)
    ref, _ = orc.split(X64, e, s, b)
    de = torch.empty(R, dtype=torch.int32, device="cuda")
    alp.alp_emul_exponents_f32(R, K, torch.from_numpy(X).cuda(), K, 0, de)
    torch.cuda.synchronize()
    assert np.array_equal(de.cpu().numpy(), e)
    out = torch.full((s, R, kpad), 7.0, dtype=torch.bfloat16, device="cuda")
    alp.alp_emul_split_f32(R, K, torch.from_numpy(X).cuda(), K, 0, de, s, k, out, kpad)
    got = out.float().cpu().numpy()
    assert np.array_equal(got[:, :, :K], ref.astype(np.float32)) and np.all(got[:, :, K:] == 0)
    XT = np.ascontiguousarray(X.T)
    df = torch.empty(R, dtype=torch.int32, device="cuda")
    alp.alp_emul_exponents_f32(R, K, torch.from_numpy(XT).cuda(), R, 1, df)
    out2 = torch.full((s, R, kpad), 7.0, dtype=torch.bfloat16, device="cuda")
    alp.alp_emul_split_f32(R, K, torch.from_numpy(XT).cuda(), R, 1, df, s, k, out2, kpad)
    torch.cuda.synchronize()
    assert np.array_equal(df.cpu().numpy(), e)
    assert np.array_equal(out2.float().cpu().numpy()[:, :, :K], ref.astype(np.float32))


def test_emul_f32_alpha_beta_padding_and_special_cases(alp, orc):
    M, N, K = 100, 70, 90
    A, B, C = f32(*inputs.gemm_operands(4300, M, N, K))
    got, _, _, full = run_emul_f32(alp, A, B, C, -2.0, 0.25, 3, lda=K + 3, ldc=N + 5)
    ref, _ = model(orc, -2.0, A, B, 0.25, C, 3, "b8")
    assert np.array_equal(got, ref)
    assert np.all(np.isnan(full[:, N:]))                     # padding of C untouched
    nanA = np.full_like(A, np.nan)
    got, _, _, _ = run_emul_f32(alp, nanA, B, C, 0.0, 0.5, 3)
    assert np.array_equal(got, np.float32(0.5) * C)
    got, _, _, _ = run_emul_f32(alp, A, B, None, 1.0, 0.0, 3)
    ref, _ = model(orc, 1.0, A, B, 0.0, None, 3, "b8")
    assert np.array_equal(got, ref)
    A[3, 4] = np.inf
    _, st, err, _ = run_emul_f32(alp, A, B, C, 1.0, 0.0, 3)
    assert st == alp.ALP_OK and err == alp.ALP_ERR_UNSUPPORTED
    ok = lambda *a: alp.alp_gemm_f32_emul(4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, *a, None, 0,
                                          stream=0, raise_on_error=False)
    assert ok(5, alp.ALP_SLICE_BF16_B8) == alp.ALP_ERR_INVALID_ARG         # s b > 32
    assert ok(1, alp.ALP_SLICE_BF16_B8) == alp.ALP_ERR_INVALID_ARG
    assert ok(3, alp.ALP_SLICE_INT8) == alp.ALP_ERR_UNSUPPORTED
    assert ok(3, alp.ALP_SLICE_BF16_B8) == alp.ALP_ERR_WORKSPACE
    assert alp.alp_gemm_f32_emul(4, 4, 4, 1.0, 6, 4, 8, 4, 0.0, 8, 4, 3, alp.ALP_SLICE_BF16_B8,
                                 None, 0, stream=0, raise_on_error=False) == alp.ALP_ERR_INVALID_ARG


def test_emul_f32_error_no_worse_than_vendor_fp32(alp, orc):
    """M = N = K = 2048, u in [-1,1): three 8-bit slices against the long-double
    product on sampled rows, next to the vendor library's FP32 GEMM (TF32 off)
    on the same float inputs: componentwise relative to |A||B| and normwise."""
    import torch
    n = 2048
    A, B, _ = inputs.gemm_operands(inputs.workload_seed("emul_8192"), n, n, n, with_c=False)
    A, B = f32(A, B)
    rows = np.arange(0, n, 128)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = orc.gemm(1.0, A64, B64, 0.0, rows=rows)
    absAB = orc.absgemm(A64, B64, rows=rows)
    got, _, err, _ = run_emul_f32(alp, A, B, None, 1.0, 0.0, 3)
    assert err == alp.ALP_OK
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        vend = (torch.from_numpy(A).cuda() @ torch.from_numpy(B).cuda()).cpu().numpy()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    u = 2.0 ** -24

    def errs(x):
        d = np.abs(x[rows].astype(np.float64) - ref)
        return float(np.max(d / absAB)) / u, float(np.linalg.norm(d) / np.linalg.norm(ref))
    e_emul, e_vend = errs(got), errs(vend)
    print({"emul_f32": e_emul, "vendor_f32": e_vend})
    assert e_emul[0] <= e_vend[0] and e_emul[1] <= e_vend[1]
    assert e_emul[0] < 0.6                       # within about half an ulp of |A||B|


def test_emul_f32_full_size_sampled_rows(alp, orc):
    """M = N = K = 8192 float, the bench's launch configuration: sampled rows
    bit-exact against the model."""
    n = 8192
    A, B, _ = inputs.gemm_operands(inputs.workload_seed("emul_8192"), n, n, n, kind="scaled",
                                   phi=4, with_c=False)
    A, B = f32(A, B)
    got, st, err, _ = run_emul_f32(alp, A, B, None, 1.0, 0.0, 3)
    assert err == alp.ALP_OK
    rows = np.array([0, 4097, 8191])
    ref, _ = model(orc, 1.0, A, B, 0.0, None, 3, "b8", rows=rows)
    assert np.array_equal(got[rows], ref)


@pytest.mark.parametrize("ta,tb", [(0, 1), (1, 0), (1, 1)])
def test_emul_f32_transposed_operands_bit_exact(alp, orc, ta, tb):
    import torch
    M, N, K = 257, 300, 333
    A, B, C = f32(*inputs.gemm_operands(4500 + 2 * ta + tb, M, N, K, kind="scaled", phi=4))
    As = np.ascontiguousarray(A.T) if ta else A
    Bs = np.ascontiguousarray(B.T) if tb else B
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (As, Bs, C))
    ws = alp.alp_gemm_f32_emul_workspace(M, N, K, 3, alp.ALP_SLICE_BF16_B8)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    alp.alp_gemm_f32_emul_ex(ta, tb, M, N, K, 1.5, dA, As.shape[1], dB, Bs.shape[1], 0.5, dC, N,
                             3, alp.ALP_SLICE_BF16_B8, work, ws)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    ref, _ = model(orc, 1.5, A, B, 0.5, C, 3, "b8")
    assert np.array_equal(dC.cpu().numpy(), ref)


@pytest.mark.parametrize("N", [1, 3, 37])
def test_recombine_f32_tight_rows(alp, N):
    """alp_emul_recombine_f32 on group sums whose rows are exactly N int32
    (the element-by-element path; the buffer ends with the last row): the
    same results as the same sums in rows padded to 256 columns."""
    import torch
    s, M = 3, 5
    kind = alp.ALP_SLICE_BF16_B8
    rng = np.random.default_rng(17 + N)
    tight = rng.integers(-2 ** 20, 2 ** 20, size=(s, M, N), dtype=np.int32)
    padded = np.zeros((s, M, 256), dtype=np.int32)
    padded[:, :, :N] = tight
    e = torch.tensor([0, 3, -5, 7, 1], dtype=torch.int32, device="cuda")
    f = torch.from_numpy(np.arange(N, dtype=np.int32) % 3 - 1).cuda()
    C0 = torch.from_numpy(rng.standard_normal((M, N)).astype(np.float32)).cuda()
    out = []
    for G, ld in ((tight, N), (padded, 256)):
        C = C0.clone()
        alp.alp_emul_recombine_f32(M, N, s, kind, torch.from_numpy(np.ascontiguousarray(G)).cuda(),
                                   ld, e, f, 1.5, 0.5, C, N)
        torch.cuda.synchronize()
        out.append(C.cpu().numpy())
    assert alp.alp_get_device_error() == alp.ALP_OK
    assert np.array_equal(out[0], out[1]) and np.all(np.isfinite(out[0]))
