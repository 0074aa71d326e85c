"""Parity of the modular emulated FP64 GEMM (alp_slice_kind ALP_SLICE_BF16_CRT,
through the C-ABI) with the oracle's plain definition of it: operands rounded
to k-bit integers per row and column, their exact product, one rounding.  The
GPU reaches that product through residues and the Chinese remainder theorem,
which the oracle never uses, so agreement bit for bit checks the residues, the
tensor-core sums and the reconstruction together.  Stage tests check each of
those against integer arithmetic done here in Python."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs

from .gpu_util import dev

pytestmark = pytest.mark.gpu

CRT = 4                                  # ALP_SLICE_BF16_CRT
# the moduli in the order the ABI documents them
MODULI = [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193]


def crt_k(K, n):
    """Largest k <= 60 with K 2^(2k+1) <= Mn (1 - 2^-18), Mn = m_1 ... m_n."""
    Mn = 1
    for m in MODULI[:n]:
        Mn *= m
    for k in range(60, 0, -1):
        if max(K, 1) * 2 ** (2 * k + 1) <= Mn - (Mn >> 18):
            return k
    return 0


def crt_weights(n):
    """y_l = (Mn / m_l)^-1 mod m_l, the weight of residue l."""
    Mn = 1
    for m in MODULI[:n]:
        Mn *= m
    return [pow(Mn // m % m, -1, m) for m in MODULI[:n]]


def run_crt(alp, A, B, C, alpha, beta, n, lda=None, ldc=None, raise_on_error=True):
    import torch
    M, K = A.shape
    N = B.shape[1]
    dA, lda = dev(A, lda)
    dB, ldb = dev(B)
    dC, ldc = dev(C if C is not None else np.full((M, N), np.nan), ldc)
    ws = alp.alp_gemm_f64_emul_workspace(M, N, K, n, CRT)
    work = torch.empty(max(ws, 1), dtype=torch.uint8, device="cuda")
    st = alp.alp_gemm_f64_emul(M, N, K, alpha, dA, lda, dB, ldb, beta, dC, ldc, n, CRT, work, ws,
                               raise_on_error=raise_on_error)
    torch.cuda.synchronize()
    return dC.cpu().numpy()[:M, :N], st, alp.alp_get_device_error()


SHAPES = [(128, 256, 64), (200, 300, 130), (1, 1, 1), (257, 513, 1000), (64, 40, 2049)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("n,phi", [(4, 0), (8, 4), (14, 0), (15, 8), (16, 0), (16, 32)])
def test_crt_bit_exact_vs_oracle(alp, orc, shape, n, phi):
    M, N, K = shape
    A, B, C = inputs.gemm_operands(5100 + M + N + K + n + phi, M, N, K, kind="scaled", phi=phi)
    got, st, err = run_crt(alp, A, B, C, 1.5, 0.5, n)
    assert st == alp.ALP_OK and err == alp.ALP_OK
    ref, rc = orc.crt_gemm(1.5, A, B, 0.5, C, crt_k(K, n))
    assert rc == 0
    assert np.array_equal(got, ref)


EDGE_ROWS = np.array([0, 1, 63, 127, 128, 129])


@pytest.mark.parametrize("K", [63, 64, 65, 1023, 1024, 1025, 2049, 8193])
def test_crt_chunk_boundaries(alp, orc, K):
    """K around the 1024-wide drain chunks and the 64-wide k-blocks."""
    M, N = 130, 260
    A, B, _ = inputs.gemm_operands(5200 + K, M, N, K, kind="scaled", phi=4, with_c=False)
    got, _, err = run_crt(alp, A, B, None, 1.0, 0.0, 15)
    assert err == alp.ALP_OK
    ref, _ = orc.crt_gemm(1.0, A, B, 0.0, None, crt_k(K, 15), rows=EDGE_ROWS)
    assert np.array_equal(got[EDGE_ROWS], ref)


@pytest.mark.parametrize("n", [4, 15])
def test_crt_partial_sums_at_the_chunk_bound(alp, orc, n):
    """Entries x = 1/2 + 2^(7-k): x 2^k = 2^(k-1) + 128, whose residue modulo
    256 is -128 for either sign, so every product of the first modulus is 2^14
    and each 1024-wide chunk's f32 partial sum is exactly 2^24, the largest the
    chunking allows; two chunks make the int32 sum 2^25."""
    K = 2048
    k = crt_k(K, n)
    x = 0.5 + 2.0 ** (7 - k)
    M, N = 130, 260
    A = np.full((M, K), x)
    A[1::2] *= -1
    B = np.full((K, N), x)
    B[:, 1::4] *= -1
    got, _, err = run_crt(alp, A, B, None, 1.0, 0.0, n)
    assert err == alp.ALP_OK
    ref, _ = orc.crt_gemm(1.0, A, B, 0.0, None, k, rows=EDGE_ROWS)
    assert np.array_equal(got[EDGE_ROWS], ref)


def test_crt_largest_k_and_modulus_count(alp, orc):
    """The largest K, 65472 (1023 k-blocks), with 16 moduli (k = 54, |P| up
    to 2^124, 1024 jobs per tile) and with 4 (k = 7)."""
    M, N, K = 130, 260, 65472
    A, B, _ = inputs.gemm_operands(5300, M, N, K, kind="scaled", phi=2, with_c=False)
    for n in (16, 4):
        got, st, err = run_crt(alp, A, B, None, 1.0, 0.0, n)
        assert st == alp.ALP_OK and err == alp.ALP_OK
        ref, _ = orc.crt_gemm(1.0, A, B, 0.0, None, crt_k(K, n), rows=EDGE_ROWS)
        assert np.array_equal(got[EDGE_ROWS], ref)
    # opposite-sign operands at their largest: |A'| = |B'| = 2^54 - 2, |P| near
    # K 2^108 = 2^124, just under Mn / 2
    A = np.ones((M, K)) * (1.0 - 2.0 ** -53)
    B = -np.ones((K, N)) * (1.0 - 2.0 ** -53)
    got, _, err = run_crt(alp, A, B, None, 1.0, 0.0, 16)
    assert err == alp.ALP_OK
    ref, _ = orc.crt_gemm(1.0, A, B, 0.0, None, crt_k(K, 16), rows=EDGE_ROWS)
    assert np.array_equal(got[EDGE_ROWS], ref) and abs(ref[0, 0] + K) <= K * 2.0 ** -50


def test_crt_alpha_beta_padding_special_cases_and_limits(alp, orc):
    import torch
    M, N, K = 100, 70, 90
    A, B, C = inputs.gemm_operands(5400, M, N, K)
    A[5] = 0.0                                       # a zero row
    B[:, 7] = 0.0                                    # a zero column
    A[6, :3] = [2.0 ** 900, -2.0 ** 850, 2.0 ** -900]
    B[:2, 8] = [2.0 ** -1000, 3.0 * 2.0 ** -1040]    # a column of tiny values
    k = crt_k(K, 15)
    got, _, err = run_crt(alp, A, B, C, -2.0, 0.25, 15, lda=K + 3, ldc=N + 5)
    assert err == alp.ALP_OK
    ref, _ = orc.crt_gemm(-2.0, A, B, 0.25, C, k)
    assert np.array_equal(got, ref)
    got, _, _ = run_crt(alp, A, B, None, 1.0, 0.0, 15)
    ref, _ = orc.crt_gemm(1.0, A, B, 0.0, None, k)
    assert np.array_equal(got, ref)
    got, _, _ = run_crt(alp, np.full_like(A, np.nan), B, C, 0.0, 0.5, 15)
    assert np.array_equal(got, 0.5 * C)
    A[3, 4] = np.inf
    _, st, err = run_crt(alp, A, B, C, 1.0, 0.0, 15)
    assert st == alp.ALP_OK and err == alp.ALP_ERR_UNSUPPORTED
    call = lambda M_, K_, n, kind=CRT: alp.alp_gemm_f64_emul(  # noqa: E731
        M_, 4, K_, 1.0, 8, K_, 8, 4, 0.0, 8, 4, n, kind, 256, 1 << 40, stream=0,
        raise_on_error=False)
    assert call(4, 4, 3) == alp.ALP_ERR_INVALID_ARG
    assert call(4, 4, 17) == alp.ALP_ERR_INVALID_ARG
    assert call(4, 65473, 16) == alp.ALP_ERR_UNSUPPORTED
    assert alp.alp_gemm_f64_emul_workspace(4, 4, 4, 3, CRT) == 0
    assert alp.alp_gemm_f64_emul_workspace(4, 4, 4, 16, CRT) > 0
    assert alp.alp_gemm_f32_emul_workspace(4, 4, 4, 4, CRT) == 0
    assert alp.alp_gemm_f32_emul(4, 4, 4, 1.0, 8, 4, 8, 4, 0.0, 8, 4, 4, CRT, 256, 1 << 40,
                                 stream=0, raise_on_error=False) == alp.ALP_ERR_UNSUPPORTED
    G = torch.zeros((15, 4, 256), dtype=torch.int32, device="cuda")
    e = torch.zeros(4, dtype=torch.int32, device="cuda")
    C4 = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    assert alp.alp_emul_recombine(4, 4, 15, CRT, G, 256, e, e, 1.0, 0.0, C4, 4,
                                  raise_on_error=False) == alp.ALP_ERR_INVALID_ARG


@pytest.mark.parametrize("n", [4, 8, 14])
def test_crt_split_rounding_at_the_range_ends(alp, orc, n):
    """k <= 51 (here 4, 8 or 14 moduli): the split rounds a 2^(k - e) by one
    FP64 fma when 2^(k - e) is a normal double, else from the IEEE fields.
    Rows at the top of the range (entries near the largest double, scale
    2^(k - 1024)), rows of tiny entries (scale up to 2^1023), rows of
    subnormals (scale beyond 2^1023: the field path), exact ties at the units
    of the scaled value, and a column of subnormals: bit-exact against the
    oracle's definition, and the residues are those of Python's integers."""
    import torch
    M, N, K = 40, 300, 200
    k = crt_k(K, n)
    assert k <= 51
    rng = np.random.default_rng(8000 + n)
    A = rng.uniform(-1, 1, (M, K))
    B = rng.uniform(-1, 1, (K, N))
    A[0] = rng.uniform(-1, 1, K) * 1.7976931348623157e308        # e = 1024
    A[1] = rng.uniform(-1, 1, K) * 2.0 ** -1000                  # scale 2^(k + 1000)
    A[2] = rng.integers(-4, 5, K) * 5e-324                       # subnormal row
    A[3] = np.ldexp(2 * rng.integers(-2 ** 20, 2 ** 20, K) + 1.0, -k - 1)   # ties
    A[3, 0] = 1.0 - 2.0 ** -53                                   # rounds up to 2^k
    A[4] = rng.uniform(-1, 1, K) * 2.0 ** (-1022 - k + 30)       # scale 2^1023 - ...
    B[:, 5] = rng.integers(-3, 4, K) * 5e-324                    # subnormal column
    B[:, 6] = rng.uniform(-1, 1, K) * 2.0 ** 1000
    got, st, err = run_crt(alp, A, B, None, 1.0, 0.0, n)
    assert st == alp.ALP_OK and err == alp.ALP_OK
    ref, rc = orc.crt_gemm(1.0, A, B, 0.0, None, k)
    assert rc == 0 and np.array_equal(got, ref)
    # the residues of the crafted rows, against exact integers formed here
    e, _ = orc.row_exponents(A)
    kpad = (K + 63) // 64 * 64
    dA = torch.from_numpy(A).cuda()
    de = torch.from_numpy(e).cuda()
    da = torch.zeros((n, M, kpad), dtype=torch.bfloat16, device="cuda")
    alp.alp_emul_split(M, K, dA, K, 0, de, n, CRT, da, kpad)
    torch.cuda.synchronize()
    ra = da.float().cpu().numpy().astype(np.int64)
    for i in range(6):
        ints = [round(Fraction(float(a)) * Fraction(2) ** (k - int(e[i]))) for a in A[i]]
        for l in range(n):
            check_residues(ra[l, i, :K], np.array(ints, dtype=object), MODULI[l])


@pytest.mark.parametrize("ta,tb", [(0, 1), (1, 0), (1, 1)])
def test_crt_transposed_operands_bit_exact(alp, orc, ta, tb):
    import torch
    M, N, K = 3 * 128 + 5, 2 * 256 + 9, 700
    A, B, C = inputs.gemm_operands(5500 + 2 * ta + tb, M, N, K, kind="scaled", phi=8)
    As = np.ascontiguousarray(A.T) if ta else A
    Bs = np.ascontiguousarray(B.T) if tb else B
    lda, ldb = As.shape[1] + 3, Bs.shape[1] + 5
    dA = torch.full((As.shape[0], lda), float("nan"), dtype=torch.float64, device="cuda")
    dA[:, :As.shape[1]] = torch.from_numpy(As)
    dB = torch.full((Bs.shape[0], ldb), float("nan"), dtype=torch.float64, device="cuda")
    dB[:, :Bs.shape[1]] = torch.from_numpy(Bs)
    dC = torch.from_numpy(C).cuda()
    ws = alp.alp_gemm_f64_emul_workspace(M, N, K, 15, CRT)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    alp.alp_gemm_f64_emul_ex(ta, tb, M, N, K, 1.5, dA, lda, dB, ldb, 0.5, dC, N, 15, CRT, work, ws)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    ref, _ = orc.crt_gemm(1.5, A, B, 0.5, C, crt_k(K, 15))
    assert np.array_equal(dC.cpu().numpy(), ref)


def scaled_ints(orc, X, k, by_rows=True):
    """X' = nearest integer (ties to even) to X 2^(k - e) per row (or column)."""
    if by_rows:
        e, _ = orc.row_exponents(X)
        return np.rint(np.ldexp(X, (k - e[:, None]).astype(np.int32))).astype(np.int64), e
    f, _ = orc.col_exponents(X)
    return np.rint(np.ldexp(X, (k - f[None, :]).astype(np.int32))).astype(np.int64), f


def residue(x, m):
    """x mod m moved to [-m/2, m/2)."""
    r = np.mod(x, m)
    return np.where(2 * r >= m + (m & 1), r - m, r)


def check_residues(r, x, m):
    """The split's residues: r = x (mod m) with |r| <= 128 (the tensor-core
    stage's bound), the representative nearest to zero or one modulus off it
    (the f32 path's quotient may round the other way within 0.003 of a tie)."""
    r = np.asarray(r, dtype=np.int64)
    near = residue(np.asarray(x, dtype=object), m).astype(np.int64)
    assert np.all(np.abs(r) <= 128)
    assert np.all((r == near) | (np.abs(r - near) == m))


@pytest.mark.parametrize("M,K,ldx_extra,n", [(100, 1100, 0, 15), (37, 8193, 1, 13),
                                              (5, 63, 3, 16), (300, 2048, 0, 4)])
def test_crt_scan_split_rows_matches_the_two_stages(alp, M, K, ldx_extra, n):
    """alp_emul_scan_split_rows (the row scan inside the row split, the GEMM's
    path for A) against alp_emul_exponents + alp_emul_split: the same
    exponents and residue planes bit for bit, on ragged and odd K, a row
    stride that breaks 16-byte alignment (ldx odd), zero, tiny and huge rows;
    an Inf is reported."""
    import torch
    rng = np.random.default_rng(6100 + M + K)
    ldx = K + ldx_extra
    X = np.zeros((M, ldx))
    X[:, :K] = rng.uniform(-1, 1, (M, K)) * np.ldexp(1.0, rng.integers(-20, 21, (M, K)))
    X[0, :K] = 0.0
    X[1 % M, :K] *= 2.0 ** -1000
    X[2 % M, :K] *= 2.0 ** 900
    kpad = (K + 63) // 64 * 64
    dX = torch.from_numpy(X).cuda()
    e1 = torch.empty(M, dtype=torch.int32, device="cuda")
    e2 = torch.empty(M, dtype=torch.int32, device="cuda")
    o1 = torch.full((n, M, kpad), 5.0, dtype=torch.bfloat16, device="cuda")
    o2 = torch.full((n, M, kpad), 7.0, dtype=torch.bfloat16, device="cuda")
    alp.alp_emul_exponents(M, K, dX, ldx, 0, e1)
    alp.alp_emul_split(M, K, dX, ldx, 0, e1, n, CRT, o1, kpad)
    alp.alp_emul_scan_split_rows(M, K, dX, ldx, e2, n, CRT, o2, kpad)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    assert torch.equal(e1, e2)
    assert torch.equal(o1.view(torch.int16), o2.view(torch.int16))
    X[M // 2, K // 2] = np.inf
    dX = torch.from_numpy(X).cuda()
    alp.alp_emul_scan_split_rows(M, K, dX, ldx, e2, n, CRT, o2, kpad)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_ERR_UNSUPPORTED
    st = alp.alp_emul_scan_split_rows(M, K, dX, ldx, e2, n, alp.ALP_SLICE_BF16, o2, kpad,
                                      raise_on_error=False)
    assert st == alp.ALP_ERR_INVALID_ARG


@pytest.mark.parametrize("n,phi", [(15, 0), (16, 8), (4, 32)])
def test_crt_split_and_slice_products_stages(alp, orc, n, phi):
    """alp_emul_split with the modular kind writes the residues of the scaled
    integers (rows of A; columns of B via trans = 1); alp_emul_slice_products
    writes the byte ((sum_k a_l b_l) y_l) mod m_l = (P y_l) mod m_l;
    alp_emul_recombine_crt turns those into the oracle's result."""
    import torch
    M, N, K = 200, 300, 1100
    kpad = (K + 63) // 64 * 64
    A, B, C = inputs.gemm_operands(5600 + n + phi, M, N, K, kind="scaled", phi=phi)
    A[0, :6] = [0.5, -0.5, 0.75, 2.0 ** -60, -(1.0 - 2.0 ** -53), 0.0]
    k = crt_k(K, n)
    Ai, e = scaled_ints(orc, A, k)
    Bi, f = scaled_ints(orc, B, k, by_rows=False)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    de = torch.from_numpy(e).cuda()
    df = torch.from_numpy(f).cuda()
    da = torch.full((n, M, kpad), 7.0, dtype=torch.bfloat16, device="cuda")
    db = torch.full((n, N, kpad), 7.0, dtype=torch.bfloat16, device="cuda")
    alp.alp_emul_split(M, K, dA, K, 0, de, n, CRT, da, kpad)
    alp.alp_emul_split(N, K, dB, N, 1, df, n, CRT, db, kpad)
    torch.cuda.synchronize()
    ra = da.float().cpu().numpy().astype(np.int64)
    rb = db.float().cpu().numpy().astype(np.int64)
    for l in range(n):
        check_residues(ra[l, :, :K], Ai, MODULI[l])
        check_residues(rb[l, :, :K], Bi.T, MODULI[l])
    assert np.all(ra[:, :, K:] == 0) and np.all(rb[:, :, K:] == 0)
    ldg = (N + 255) // 256 * 256
    G = torch.full((n, M, ldg), 255, dtype=torch.uint8, device="cuda")
    alp.alp_emul_slice_products(M, N, K, n, CRT, da, db, kpad, G, ldg)
    torch.cuda.synchronize()
    g = G.cpu().numpy()
    y = crt_weights(n)
    for l in range(n):
        Q = ra[l, :, :K] @ rb[l, :, :K].T
        assert np.abs(Q).max() <= K * 2 ** 14
        assert np.array_equal(g[l, :, :N], np.mod(np.mod(Q, MODULI[l]) * y[l], MODULI[l])), l
    dC = torch.from_numpy(C.copy()).cuda()
    alp.alp_emul_recombine_crt(M, N, K, n, G, ldg, de, df, 1.5, 0.5, dC, N)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    ref, _ = orc.crt_gemm(1.5, A, B, 0.5, C, k)
    assert np.array_equal(dC.cpu().numpy(), ref)


@pytest.mark.parametrize("cfg", [None, (256, 256, 64, 2, 0, 1), (128, 256, 64, 1, 0, 8)])
@pytest.mark.parametrize("M,N,K,n", [(1000, 1300, 700, 15), (3 * 256 + 1, 5 * 256 - 3, 2100, 13),
                                     (64, 2000, 300, 16), (300, 200, 5000, 14)])
def test_crt_gemm_call_matches_its_stages(alp, orc, cfg, M, N, K, n):
    """The GEMM call for both block arrangements, on shapes whose last wave is
    cut into pieces by moduli and on ragged ones: bit-exact against the
    oracle's definition on rows across tile edges, and equal element for
    element to its stages run one by one through the C-ABI (exponents,
    splits, alp_emul_slice_products, alp_emul_recombine_crt)."""
    import torch
    A, B, C = inputs.gemm_operands(5900 + M + N + n, M, N, K, kind="scaled", phi=3)
    if cfg is not None:
        alp.alp_tune_set_cached(M, N, K, alp.ALP_PATH_EMUL, cfg)
    try:
        got, st, err = run_crt(alp, A, B, C, -1.0, 0.25, n)
    finally:
        alp.alp_tune_clear_cache()
    assert st == alp.ALP_OK and err == alp.ALP_OK
    rows = np.unique(np.clip([0, 1, 127, 128, 129, 255, 256, 257, M // 2, M - 2, M - 1], 0, M - 1))
    ref, rc = orc.crt_gemm(-1.0, A, B, 0.25, C, crt_k(K, n), rows=rows)
    assert rc == 0 and np.array_equal(got[rows], ref)
    kpad = (K + 63) // 64 * 64
    ldg = (N + 255) // 256 * 256
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    de = torch.empty(M, dtype=torch.int32, device="cuda")
    df = torch.empty(N, dtype=torch.int32, device="cuda")
    alp.alp_emul_exponents(M, K, dA, K, 0, de)
    alp.alp_emul_exponents(N, K, dB, N, 1, df)
    da = torch.empty((n, M, kpad), dtype=torch.bfloat16, device="cuda")
    db = torch.empty((n, N, kpad), dtype=torch.bfloat16, device="cuda")
    alp.alp_emul_split(M, K, dA, K, 0, de, n, CRT, da, kpad)
    alp.alp_emul_split(N, K, dB, N, 1, df, n, CRT, db, kpad)
    G = torch.full((n, M, ldg), 255, dtype=torch.uint8, device="cuda")
    alp.alp_emul_slice_products(M, N, K, n, CRT, da, db, kpad, G, ldg)
    dC = torch.from_numpy(C.copy()).cuda()
    alp.alp_emul_recombine_crt(M, N, K, n, G, ldg, de, df, -1.0, 0.25, dC, N)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    assert np.array_equal(got, dC.cpu().numpy())


@pytest.mark.parametrize("M,N,K,n,alpha,beta", [
    (2560, 2560, 300, 15, 1.0, 0.0),      # one whole tile per CTA pair, then a tail piece
    (4096, 4100, 200, 16, -1.0, 0.5),     # several whole tiles per pair, ragged columns
    (3000, 1500, 1100, 13, 0.75, -2.0),   # ragged rows, chunks of two lengths
    (300, 200, 700, 4, 1.0, 1.0),         # every tile in the tail
    (256 * 76, 256, 64, 14, 1.0, 0.0)])   # one tile per pair, no tail when 76 pairs fit
def test_crt_products_recombine_matches_the_two_stages(alp, orc, M, N, K, n, alpha, beta):
    """alp_emul_products_recombine_crt (the tensor-core stage with the
    reconstruction of each tile in its epilogue, the persistent launch and
    the tail tiles' launch) writes the same byte planes and the same C as
    alp_emul_slice_products followed by alp_emul_recombine_crt, element for
    element, and C matches the oracle on rows across tile edges."""
    import torch
    A, B, C = inputs.gemm_operands(6100 + M + N + n, M, N, K, kind="scaled", phi=2)
    kpad = (K + 63) // 64 * 64
    ldg = (N + 255) // 256 * 256
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    de = torch.empty(M, dtype=torch.int32, device="cuda")
    df = torch.empty(N, dtype=torch.int32, device="cuda")
    alp.alp_emul_exponents(M, K, dA, K, 0, de)
    alp.alp_emul_exponents(N, K, dB, N, 1, df)
    da = torch.empty((n, M, kpad), dtype=torch.bfloat16, device="cuda")
    db = torch.empty((n, N, kpad), dtype=torch.bfloat16, device="cuda")
    alp.alp_emul_split(M, K, dA, K, 0, de, n, CRT, da, kpad)
    alp.alp_emul_split(N, K, dB, N, 1, df, n, CRT, db, kpad)
    G1 = torch.full((n, M, ldg), 255, dtype=torch.uint8, device="cuda")
    C1 = torch.from_numpy(C.copy()).cuda()
    wsb = alp.alp_emul_products_recombine_crt_workspace(M, N)
    work = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    alp.alp_emul_products_recombine_crt(M, N, K, n, da, db, kpad, G1, ldg, de, df, alpha, beta,
                                        C1, N, work, wsb)
    G2 = torch.full((n, M, ldg), 255, dtype=torch.uint8, device="cuda")
    C2 = torch.from_numpy(C.copy()).cuda()
    alp.alp_emul_slice_products(M, N, K, n, CRT, da, db, kpad, G2, ldg)
    alp.alp_emul_recombine_crt(M, N, K, n, G2, ldg, de, df, alpha, beta, C2, N)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    assert torch.equal(G1[:, :, :N], G2[:, :, :N])
    got = C1.cpu().numpy()
    assert np.array_equal(got, C2.cpu().numpy())
    rows = np.unique(np.clip([0, 127, 128, 255, 256, 511, 512, M // 2, M - 1], 0, M - 1))
    ref, rc = orc.crt_gemm(alpha, A, B, beta, C, crt_k(K, n), rows=rows)
    assert rc == 0 and np.array_equal(got[rows], ref)


_FUSE_CHILD = """
import sys, numpy as np, torch
from paper_1706_10086_gb300 import alp, inputs
M, N, K, n = 1300, 900, 700, 15
A, B, C = inputs.gemm_operands(6400, M, N, K, kind="scaled", phi=3)
dA, dB, dC = (torch.from_numpy(x.copy()).cuda() for x in (A, B, C))
ws = alp.alp_gemm_f64_emul_workspace(M, N, K, n, alp.ALP_SLICE_BF16_CRT)
work = torch.empty(ws, dtype=torch.uint8, device="cuda")
alp.alp_gemm_f64_emul(M, N, K, -0.5, dA, K, dB, N, 2.0, dC, N, n, alp.ALP_SLICE_BF16_CRT, work, ws)
torch.cuda.synchronize()
assert alp.alp_get_device_error() == alp.ALP_OK
np.save(sys.argv[1], dC.cpu().numpy())
"""


def test_crt_fuse_switch_gives_the_same_result(tmp_path):
    """alp_gemm_f64_emul's modular scheme with ALP_EMUL_CRT_FUSE=0 (the
    products, then the reconstruction kernel) and with the default fused
    launch write the same C, element for element (child processes: the switch
    is read once per process)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for fuse in ("1", "0"):
        path = str(tmp_path / f"c_{fuse}.npy")
        env = dict(os.environ, ALP_EMUL_CRT_FUSE=fuse)
        subprocess.run([sys.executable, "-c", _FUSE_CHILD, path], cwd=root, env=env,
                       check=True, timeout=600)
        out[fuse] = np.load(path)
    assert np.array_equal(out["1"], out["0"])


def test_crt_products_recombine_argument_errors(alp):
    """The fused stage rejects what the two stages reject, and K < 1, and a
    missing or short schedule workspace, before any launch."""
    import torch
    # every buffer holds what a 64 x 300 x 128 call with 16 moduli would touch
    d = torch.zeros(1 << 18, dtype=torch.float64, device="cuda")
    e = torch.zeros(512, dtype=torch.int32, device="cuda")
    wsb = alp.alp_emul_products_recombine_crt_workspace(64, 300)
    assert wsb > 0 and alp.alp_emul_products_recombine_crt_workspace(0, 64) == 0
    w = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    bad = [(64, 64, 0, 15, 64, 256), (64, 64, 64, 3, 64, 256), (64, 64, 64, 17, 64, 256),
           (64, 64, 64, 15, 32, 256), (64, 64, 100, 15, 100, 256), (64, 64, 64, 15, 64, 128),
           (64, 300, 64, 15, 64, 256)]
    for M, N, K, n, kpad, ldg in bad:
        st = alp.alp_emul_products_recombine_crt(M, N, K, n, d, d, kpad, d, ldg, e, e, 1.0, 0.0,
                                                 d, max(N, 1), w, wsb, raise_on_error=False)
        assert st == alp.ALP_ERR_INVALID_ARG, (M, N, K, n, kpad, ldg)
    st = alp.alp_emul_products_recombine_crt(64, 64, 64, 15, d, d, 64, None, 256, e, e, 1.0, 0.0,
                                             d, 64, w, wsb, raise_on_error=False)
    assert st == alp.ALP_ERR_INVALID_ARG
    need = alp.alp_emul_products_recombine_crt_workspace(64, 64)
    for work, nb in ((None, need), (w, need - 4)):
        st = alp.alp_emul_products_recombine_crt(64, 64, 64, 15, d, d, 64, d, 256, e, e, 1.0, 0.0,
                                                 d, 64, work, nb, raise_on_error=False)
        assert st == alp.ALP_ERR_WORKSPACE
    assert alp.alp_get_device_error() == alp.ALP_OK


@pytest.mark.parametrize("n", list(range(4, 17)))
def test_crt_recombine_rounding(alp, n):
    """alp_emul_recombine_crt on crafted residues: P anywhere in [-L, L],
    L = floor((Mn - Mn/2^18) / 2) the largest |P| the k rule admits (the
    ends included), given as the bytes (P y_l) mod m_l, with tails that are exact ties, just off a
    tie, or carry one sticky bit; each result must be the correctly rounded
    alpha-free value P 2^(e_i + f_j - 2k) (Python's exact rational rounding)."""
    import random

    import torch
    K = 8192
    k = crt_k(K, n)
    Mn = 1
    for m in MODULI[:n]:
        Mn *= m
    rnd = random.Random(33 + n)
    L = (Mn - (Mn >> 18)) // 2
    assert K * 2 ** (2 * k) <= L          # every product the k rule admits
    vals = [0, 1, -1, L, -L, L - 1, 2 ** 53 + 1, -(2 ** 54 + 2)]
    vals = [v for v in vals if abs(v) <= L]
    top = L.bit_length()
    while len(vals) < 500:
        nbits = rnd.randrange(1, top)
        X = rnd.getrandbits(nbits) | (1 << (nbits - 1))
        form = rnd.randrange(5)
        if nbits > 54 and form < 4:
            r = nbits - 54 if form < 3 else rnd.randrange(0, nbits - 54)
            X = (X >> (r + 1)) << (r + 1)
            X += [1 << r, (1 << r) - 1, (1 << r) + 1, 1 << r][form]
        if X <= L:
            vals.append(-X if rnd.random() < 0.5 else X)
    N = len(vals)
    ldg = (N + 255) // 256 * 256
    rows = 5
    G = np.zeros((n, rows, ldg), dtype=np.uint8)
    y = crt_weights(n)
    for j, P in enumerate(vals):
        for l, m in enumerate(MODULI[:n]):
            G[l, :, j] = P * y[l] % m
    # the last two rows scale mid-sized P into the subnormal range and past the
    # largest double
    e = np.array([0, 5, -40, 2 * k - 1074 - top // 2, 2 * k + 1024 - top // 2], dtype=np.int32)
    f = np.array([rnd.randrange(-8, 9) for _ in range(N)], dtype=np.int32)
    dC = torch.full((rows, N), float("nan"), dtype=torch.float64, device="cuda")
    alp.alp_emul_recombine_crt(rows, N, K, n, torch.from_numpy(G).cuda(), ldg,
                               torch.from_numpy(e).cuda(), torch.from_numpy(f).cuda(), 1.0, 0.0,
                               dC, N)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    for r in range(rows):
        for j, P in enumerate(vals):
            E = int(e[r]) + int(f[j]) - 2 * k
            if r < 3:
                want = float(Fraction(P) * Fraction(2) ** E)      # one rounding
            else:
                # the definition: P rounded to double, then scaled (a second
                # rounding below the normal range, infinity above it)
                with np.errstate(over="ignore"):
                    want = float(np.ldexp(np.float64(float(P)), E))
            assert got[r, j] == want, (r, j, P, E)
    assert np.isinf(got[4]).any() and np.isfinite(got[4]).any()
    assert ((got[3] != 0) & (np.abs(got[3]) < 2.0 ** -1022)).any()


def test_crt_host_resident_operands(alp, orc):
    """A, B and C in pageable host memory on a device that reads it through
    the host's page tables (alp_host_access): the residue splits read A and B
    there and the reconstruction writes C there; skipped elsewhere."""
    import torch
    pageable, _ = alp.alp_host_access()
    if not pageable:
        pytest.skip("this device does not access pageable host memory")
    M, N, K = 3 * 128 + 5, 2 * 256 + 9, 700
    A, B, C = inputs.gemm_operands(5700, M, N, K, kind="scaled", phi=8)
    A, B = np.ascontiguousarray(A), np.ascontiguousarray(B)
    hC = np.ascontiguousarray(C.copy())
    ws = alp.alp_gemm_f64_emul_workspace(M, N, K, 15, CRT)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    alp.alp_gemm_f64_emul(M, N, K, 1.5, A.ctypes.data, K, B.ctypes.data, N, 0.5, hC.ctypes.data,
                          N, 15, CRT, work, ws)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    ref, _ = orc.crt_gemm(1.5, A, B, 0.5, C, crt_k(K, 15))
    assert np.array_equal(hC, ref)


@pytest.mark.parametrize("N", [1, 2, 3, 37, 517])
def test_crt_recombine_tight_rows(alp, N):
    """alp_emul_recombine_crt on byte planes whose rows are exactly N bytes
    (not a multiple of 4: the byte-by-byte path), the buffer ending with the
    last row, beta != 0: the same results as the same residues in padded
    rows (the word-load path)."""
    import random

    import torch
    n, K, M = 15, 8192, 3
    k = crt_k(K, n)
    Mn = 1
    for m in MODULI[:n]:
        Mn *= m
    L = (Mn - (Mn >> 18)) // 2
    rnd = random.Random(91 + N)
    y = crt_weights(n)
    P = [rnd.randrange(-L, L + 1) for _ in range(M * N)]
    tight = np.zeros((n, M, N), dtype=np.uint8)
    for idx, p in enumerate(P):
        for l, m in enumerate(MODULI[:n]):
            tight[l, idx // N, idx % N] = p * y[l] % m
    ldp = (N + 255) // 256 * 256
    padded = np.zeros((n, M, ldp), dtype=np.uint8)
    padded[:, :, :N] = tight
    e = torch.tensor([3, -7, 0], dtype=torch.int32, device="cuda")
    f = torch.from_numpy(np.arange(N, dtype=np.int32) % 5 - 2).cuda()
    C0 = torch.from_numpy(inputs.uniform(93, 0, (M, N))).cuda()
    out = []
    for R, ld in ((tight, N), (padded, ldp)):
        C = C0.clone()
        alp.alp_emul_recombine_crt(M, N, K, n, torch.from_numpy(np.ascontiguousarray(R)).cuda(),
                                   ld, e, f, 1.5, 0.5, C, N)
        torch.cuda.synchronize()
        out.append(C.cpu().numpy())
    assert alp.alp_get_device_error() == alp.ALP_OK
    assert np.array_equal(out[0], out[1])
    for idx in (0, M * N - 1):
        i, j = divmod(idx, N)
        E = int(e[i]) + int(f[j]) - 2 * k
        w = float(Fraction(P[idx]) * Fraction(2) ** E)
        # alpha w rounded, then fma(beta, C, .) rounded once
        want = float(Fraction(0.5) * Fraction(C0[i, j].item()) + Fraction(1.5 * w))
        assert out[0][i, j] == want


def test_crt_full_size_sampled_rows(alp, orc):
    """M = N = K = 8192 in the bench's launch configuration (CTA pairs, the
    last partial wave split by moduli): sampled rows bit-exact against the
    oracle's definition for 15 moduli (phi = 0, the bench's inputs' range) and
    16 (phi = 8), with alpha = 1.5 and beta = 0.5."""
    M = N = K = 8192
    rows = np.array([0, 1, 4097, 8190, 8191])
    for n, phi in ((15, 0), (16, 8)):
        A, B, C = inputs.gemm_operands(inputs.workload_seed("emul_8192") + phi, M, N, K,
                                       kind="scaled", phi=phi)
        got, st, err = run_crt(alp, A, B, C, 1.5, 0.5, n)
        assert st == alp.ALP_OK and err == alp.ALP_OK
        ref, _ = orc.crt_gemm(1.5, A, B, 0.5, C, crt_k(K, n), rows=rows)
        assert np.array_equal(got[rows], ref), n


# ---- automatic modulus count (nslices = 0) ----

U53 = 2.0 ** -53


def _line_stats(X, e):
    """Statistics of the lines of X (rows), scale exponents e, in float64:
    x = |entry| 2^-e, S1 = sum x, S2 = sum x^2 -> (max 1/S1^2, max S2/S1^2,
    max 1/S2) over the nonzero lines."""
    x = np.abs(X) * np.ldexp(1.0, -np.asarray(e, dtype=np.int64))[:, None]
    s1, s2 = x.sum(axis=1), (x * x).sum(axis=1)
    keep = s1 > 0
    s1, s2 = s1[keep], s2[keep]
    return [float(np.max(1 / s1 ** 2)), float(np.max(s2 / s1 ** 2)), float(np.max(1 / s2))]


@pytest.mark.parametrize("phi", [0, 8, 32])
def test_crt_auto_count_no_worse_than_native(alp, orc, phi):
    """nslices = 0: the count the library picks from the operands' statistics
    gives a result bit-exact with the oracle's definition at that count, and,
    against the long-double oracle on sampled rows, a largest componentwise
    error (relative to |A||B|) and a normwise error no worse than the native
    FP64 kernel's on the same inputs, for entries u 2^e with e in [-phi, phi].
    The statistics the GPU read agree with a float64 recomputation here (the
    rule's predictions within 1e-3)."""
    import torch
    M, N, K = 512, 384, 4096
    A, B, _ = inputs.gemm_operands(7700 + phi, M, N, K, kind="scaled", phi=phi, with_c=False)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ws = alp.alp_gemm_f64_emul_workspace(M, N, K, 0, CRT)
    assert ws == alp.alp_gemm_f64_emul_workspace(M, N, K, 16, CRT)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    n, pred = alp.alp_emul_crt_choose(0, 0, M, N, K, dA, K, dB, N, work, ws)
    assert 4 <= n <= 16
    st = _line_stats(A, orc.row_exponents(A)[0]) + _line_stats(B.T, orc.col_exponents(B)[0])
    n_cpu, pred_cpu = alp.alp_emul_crt_moduli_rule(M, N, K, st)
    assert np.allclose(pred, pred_cpu, rtol=1e-3), (pred, pred_cpu)
    assert n == n_cpu
    dC = torch.empty(M, N, dtype=torch.float64, device="cuda")
    alp.alp_gemm_f64_emul(M, N, K, 1.0, dA, K, dB, N, 0.0, dC, N, 0, CRT, work, ws)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    got = dC.cpu().numpy()
    rows = np.arange(0, M, 8)
    want, rc = orc.crt_gemm(1.0, A, B, 0.0, None, crt_k(K, n), rows=rows)
    assert rc == 0 and np.array_equal(got[rows], want)
    ref = orc.gemm(1.0, A, B, 0.0, rows=rows)
    absAB = orc.absgemm(A, B, rows=rows)
    dN = torch.empty_like(dC)
    alp.alp_gemm_f64(M, N, K, 1.0, dA, K, dB, N, 0.0, dN, N)
    torch.cuda.synchronize()
    nat = dN.cpu().numpy()[rows]

    def errs(x):
        d = np.abs(x - ref)
        return float(np.max(d / absAB) / U53), float(np.linalg.norm(d) / np.linalg.norm(ref))
    e_auto, e_nat = errs(got[rows]), errs(nat)
    print({"phi": phi, "n": n, "pred": pred, "auto": e_auto, "native": e_nat})
    assert e_auto[0] <= e_nat[0] and e_auto[1] <= e_nat[1], (n, e_auto, e_nat)


@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_crt_auto_count_transposed_and_ragged(alp, orc, ta, tb):
    """The automatic count through alp_gemm_f64_emul_ex with transposed
    operands, a ragged shape and alpha/beta: the same count as
    alp_emul_crt_choose on the same storage, and bit-exact with the oracle's
    definition at that count."""
    import torch
    M, N, K = 133, 70, 517
    A, B, C = inputs.gemm_operands(7800 + 2 * ta + tb, M, N, K, kind="scaled", phi=4)
    sA = np.ascontiguousarray(A.T) if ta else A
    sB = np.ascontiguousarray(B.T) if tb else B
    dA, lda = dev(sA)
    dB, ldb = dev(sB)
    dC, ldc = dev(C)
    ws = alp.alp_gemm_f64_emul_workspace(M, N, K, 0, CRT)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    n, _ = alp.alp_emul_crt_choose(ta, tb, M, N, K, dA, lda, dB, ldb, work, ws)
    alp.alp_gemm_f64_emul_ex(ta, tb, M, N, K, 1.5, dA, lda, dB, ldb, 0.5, dC, ldc, 0, CRT, work,
                             ws)
    torch.cuda.synchronize()
    assert alp.alp_get_device_error() == alp.ALP_OK
    want, rc = orc.crt_gemm(1.5, A, B, 0.5, C, crt_k(K, n))
    assert rc == 0 and np.array_equal(dC.cpu().numpy()[:M, :N], want)
