"""Pins of the CPU oracle against facts that do not come from the oracle itself:
exact rational arithmetic (brute force), closed forms, integer arithmetic,
library routines for the special cases, and the mathematics of the digit
split.  All CPU-only."""
from fractions import Fraction
import math

import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs

U = 2.0 ** -53


def exact_gemm(alpha, A, B, beta, C):
    """alpha*A*B + beta*C in exact rationals (no rounding anywhere)."""
    M, K = A.shape
    N = B.shape[1]
    out = [[None] * N for _ in range(M)]
    fa, fb = Fraction(alpha), Fraction(beta)
    for i in range(M):
        for j in range(N):
            s = sum((Fraction(A[i, k]) * Fraction(B[k, j]) for k in range(K)), Fraction(0))
            v = fa * s
            if beta != 0.0:
                v += fb * Fraction(C[i, j])
            out[i][j] = v
    return out


def ulp(x: float) -> float:
    return math.ulp(x) if x != 0 else 2.0 ** -1074


SHAPES_TINY = [(1, 1, 1), (2, 3, 4), (3, 1, 5), (8, 8, 8), (5, 7, 3), (1, 8, 2)]
SHAPES_RESIDUE = [(17, 3, 31), (3, 33, 16), (15, 2, 33), (33, 17, 1)]


@pytest.mark.parametrize("shape", SHAPES_TINY + SHAPES_RESIDUE)
def test_gemm_matches_exact_rational(orc, shape):
    """Long-double triple loop vs exact rationals: within the rounding of the
    result plus the long-double accumulation error (never a dropped term,
    sign flip or transposed operand, which all miss by O(1))."""
    M, N, K = shape
    seed = 7000 + M * 1000 + N * 10 + K
    A, B, C = inputs.gemm_operands(seed, M, N, K)
    alpha, beta = 1.5, 0.5
    D = orc.gemm(alpha, A, B, beta, C)
    E = exact_gemm(alpha, A, B, beta, C)
    absAB = np.abs(A) @ np.abs(B)
    eps_ld = 2.0 ** (-orc.long_double_digits() + 1)
    for i in range(M):
        for j in range(N):
            ex = float(E[i][j])                # correctly rounded exact value
            err = abs(Fraction(D[i, j]) - E[i][j])
            budget = Fraction(ulp(ex)) / 2 + Fraction(
                (K + 2) * eps_ld * (abs(alpha) * absAB[i, j] + abs(beta * C[i, j])))
            assert err <= budget, (i, j, D[i, j], ex)


@pytest.mark.parametrize("shape", [(4, 5, 6), (16, 9, 33)])
def test_gemm_dyadic_inputs_exact(orc, shape):
    """Inputs with few significant bits: every operation is exact, so the
    oracle must equal the rational result exactly."""
    M, N, K = shape
    A = inputs.integers(11, 0, (M, K)) / 8.0
    B = inputs.integers(12, 0, (K, N)) / 4.0
    C = inputs.integers(13, 0, (M, N)) / 2.0
    D = orc.gemm(2.0, A, B, 0.5, C)
    E = exact_gemm(2.0, A, B, 0.5, C)
    for i in range(M):
        for j in range(N):
            assert Fraction(D[i, j]) == E[i][j]


def test_integer_config_equals_int64_matmul(orc):
    """Integer entries in {-8..8}, K = 512: every partial sum fits FP64 exactly,
    so the result equals numpy's exact int64 matrix product."""
    M, N, K = 48, 40, 512
    A, B, _ = inputs.gemm_operands(inputs.workload_seed("dgemm_512"), M, N, K, kind="int",
                                   with_c=False)
    D = orc.gemm(1.0, A, B, 0.0)
    ref = A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(D, ref.astype(np.float64))


def test_identity_and_permutation(orc):
    M = 24
    rng_perm = np.argsort(inputs.uniform(5, 0, (M,)))
    B = inputs.uniform(6, 0, (M, 17))
    C = inputs.uniform(7, 0, (M, 17))
    eye = np.eye(M)
    # A = I: C = alpha*B + beta*C (one rounding each side, long double sum exact)
    D = orc.gemm(1.0, eye, B, 0.0, C)
    assert np.array_equal(D, B)
    # A = permutation: rows of B permuted, bit for bit
    P = eye[rng_perm]
    D = orc.gemm(1.0, P, B, 0.0)
    assert np.array_equal(D, B[rng_perm])
    # alpha = 2, beta = 0.5 are powers of two: exact
    D = orc.gemm(2.0, eye, B, 0.5, C)
    assert np.array_equal(D, 2.0 * B + 0.5 * C)


def test_rank_one(orc):
    """A_ik = x_i, B_kj = y_j  =>  C_ij = alpha*K*x_i*y_j + beta*C_ij (small integers: exact)."""
    M, N, K = 9, 11, 37
    x = inputs.integers(21, 0, (M,))
    y = inputs.integers(22, 0, (N,))
    A = np.repeat(x[:, None], K, axis=1)
    B = np.repeat(y[None, :], K, axis=0)
    C = inputs.integers(23, 0, (M, N))
    D = orc.gemm(3.0, A, B, -2.0, C)
    assert np.array_equal(D, 3.0 * K * np.outer(x, y) - 2.0 * C)


def test_alpha_beta_edge_cases(orc):
    M, N, K = 6, 5, 4
    A, B, C = inputs.gemm_operands(31, M, N, K)
    # B = 0: C = beta*C
    D = orc.gemm(1.5, A, np.zeros((K, N)), 0.5, C)
    assert np.array_equal(D, 0.5 * C)
    # alpha = 0 reads neither A nor B: NaN there must not appear
    An = np.full_like(A, np.nan)
    Bn = np.full_like(B, np.nan)
    D = orc.gemm(0.0, An, Bn, 0.5, C)
    assert np.array_equal(D, 0.5 * C)
    # beta = 0 reads no C
    Cn = np.full_like(C, np.nan)
    D = orc.gemm(1.0, A, B, 0.0, Cn)
    assert not np.isnan(D).any()
    # K = 0
    D = orc.gemm(1.0, np.zeros((M, 0)), np.zeros((0, N)), 2.0, C)
    assert np.array_equal(D, 2.0 * C)


def test_row_sampling_matches_full(orc):
    M, N, K = 20, 13, 21
    A, B, C = inputs.gemm_operands(41, M, N, K)
    full = orc.gemm(1.5, A, B, 0.5, C)
    rows = np.array([19, 0, 7, 7])
    part = orc.gemm(1.5, A, B, 0.5, C, rows=rows)
    assert np.array_equal(part, full[rows])


def test_absgemm(orc):
    A, B, _ = inputs.gemm_operands(43, 7, 9, 12)
    D = orc.absgemm(A, B)
    E = exact_gemm(1.0, np.abs(A), np.abs(B), 0.0, None)
    for i in range(7):
        for j in range(9):
            assert abs(Fraction(D[i, j]) - E[i][j]) <= Fraction(ulp(float(E[i][j])))


def test_bound_holds_for_fp64_recursive_sum(orc):
    """The acceptance bound 2 K u |alpha| (|A||B|) + u |beta C| holds for a
    plain FP64 recursive summation (a textbook result, Higham Thm 3.1), here
    computed with Python floats, measured against the oracle."""
    M, N, K = 5, 6, 200
    A, B, C = inputs.gemm_operands(47, M, N, K)
    alpha, beta = 1.5, 0.5
    D = orc.gemm(alpha, A, B, beta, C)
    absAB = orc.absgemm(A, B)
    bound = orc.error_bound(alpha, absAB, beta, C, K)
    for i in range(M):
        for j in range(N):
            s = 0.0
            for k in range(K):
                s = s + A[i, k] * B[k, j]
            v = alpha * s + beta * C[i, j]
            assert abs(v - D[i, j]) <= bound[i, j]


# ---------------------------------------------------------------------------
# Emulated-GEMM model.
# ---------------------------------------------------------------------------

def test_row_exponents_follow_frexp(orc):
    A = inputs.scaled(51, 0, (9, 13), phi=20)
    A[3] = 0.0
    A[5, 4] = 2.0 ** -1070          # subnormal row maximum is fine
    A[5, :4] = 0.0
    A[5, 5:] = 0.0
    e, bad = orc.row_exponents(A)
    assert not bad
    for i in range(9):
        m = np.max(np.abs(A[i]))
        assert e[i] == (math.frexp(m)[1] if m != 0 else 0)
        if m != 0:
            assert 2.0 ** (e[i] - 1) <= m < 2.0 ** e[i]
    f, bad = orc.col_exponents(A.T.copy())
    assert np.array_equal(f, e)
    A[2, 2] = np.inf
    assert orc.row_exponents(A)[1]
    A[2, 2] = np.nan
    assert orc.row_exponents(A)[1]


@pytest.mark.parametrize("phi", [0, 8, 32])
@pytest.mark.parametrize("s,b", [(8, 7), (7, 8)])
def test_split_reconstructs_exactly(orc, phi, s, b):
    """sum_p d_p 2^(-p b) + r_s 2^(-s b) = A 2^-e exactly; digit bounds; each
    digit is the round-half-even of the exact scaled remainder."""
    A = inputs.scaled(60 + phi, 0, (6, 10), phi)
    A[0, 0] = 0.5 * 2.0 ** 3        # exact ties appear for short dyadics
    A[0, 1] = -0.75 * 2.0 ** 3
    e, _ = orc.row_exponents(A)
    d, rem = orc.split(A, e, s, b)
    for i in range(6):
        for k in range(10):
            r = Fraction(A[i, k]) / Fraction(2) ** int(e[i])
            assert abs(r) < 1
            for p in range(s):
                x = r * 2 ** b
                q = round(x)                      # Fraction.__round__: half to even
                assert d[p, i, k] == q
                assert abs(q) <= (2 ** b if p == 0 else 2 ** (b - 1))
                r = x - q
            assert Fraction(rem[i, k]) == r
            recon = sum(Fraction(int(d[p, i, k])) / Fraction(2) ** (b * (p + 1)) for p in range(s))
            recon += Fraction(rem[i, k]) / Fraction(2) ** (b * s)
            assert recon * Fraction(2) ** int(e[i]) == Fraction(A[i, k])


def emul_budget(alpha, beta, C, e, f, K, s, b, out, trim=False):
    """Error of the emulated GEMM against the exact product: cut-off digits and
    dropped pairs (<= 2^(e_i+f_j) K 2^(-s b) (1 + 0.26 s)) plus the roundings
    of the conversion, the alpha product and the beta fma (<= 3 u |out| + u |beta C|).
    The trimmed last group drops s-2 more pairs (p, q >= 2, p + q = s+1), each
    at most K 2^(2b-2) 2^(-(s+1) b) 2^(e_i+f_j)."""
    scale = np.ldexp(1.0, (e[:, None] + f[None, :]).astype(np.int64))
    t = scale * K * 2.0 ** (-s * b) * (1 + 0.26 * s) * abs(alpha)
    if trim:
        t = t + scale * K * max(s - 2, 0) * 2.0 ** (2 * b - 2 - (s + 1) * b) * abs(alpha)
    return t + 3 * U * np.abs(out) + (U * np.abs(beta * C) if beta != 0 else 0.0) + 1e-300


@pytest.mark.parametrize("s,b,trim", [(3, 7, 0), (5, 7, 0), (8, 7, 0), (3, 8, 0), (6, 8, 0),
                                      (7, 8, 0), (3, 8, 1), (5, 8, 1), (7, 8, 1)])
@pytest.mark.parametrize("phi", [0, 8])
def test_emul_gemm_within_derived_bound(orc, s, b, trim, phi):
    M, N, K = 5, 4, 23
    A, B, C = inputs.gemm_operands(70 + s + phi, M, N, K, kind="scaled", phi=phi)
    alpha, beta = 1.5, 0.5
    D, rc = orc.emul_gemm(alpha, A, B, beta, C, s, b=b, trim=trim)
    assert rc == 0
    E = exact_gemm(alpha, A, B, beta, C)
    e, _ = orc.row_exponents(A)
    f, _ = orc.col_exponents(B)
    bud = emul_budget(alpha, beta, C, e, f, K, s, b, D, trim)
    for i in range(M):
        for j in range(N):
            assert abs(Fraction(D[i, j]) - E[i][j]) <= Fraction(bud[i, j]), (i, j, s, phi)


def fraction_digits(x: float, e: int, s: int, b: int):
    """Digits of x * 2^-e by exact rational arithmetic, round half to even."""
    r = Fraction(x) / Fraction(2) ** e
    out = []
    for _ in range(s):
        y = r * 2 ** b
        q = round(y)
        out.append(q)
        r = y - q
    return out


def fraction_emul(alpha, A, B, beta, C, s, b, trim=False):
    """The emulated GEMM evaluated independently of the C oracle: digits and
    products in exact rationals, the kept sum rounded by Python's correctly
    rounded int -> float, scalings with math.ldexp, the fma in rationals.
    trim: of the pairs with p + q = s + 1 only (1, s) and (s, 1) are kept."""
    M, K = A.shape
    N = B.shape[1]
    e = [math.frexp(float(np.max(np.abs(A[i]))))[1] if np.any(A[i]) else 0 for i in range(M)]
    f = [math.frexp(float(np.max(np.abs(B[:, j]))))[1] if np.any(B[:, j]) else 0
         for j in range(N)]
    dA = [[fraction_digits(A[i, k], e[i], s, b) for k in range(K)] for i in range(M)]
    dB = [[fraction_digits(B[k, j], f[j], s, b) for k in range(K)] for j in range(N)]
    out = np.empty((M, N))
    for i in range(M):
        for j in range(N):
            X = 0
            for p in range(1, s + 1):
                for q in range(1, s + 2 - p):
                    if trim and p + q == s + 1 and min(p, q) > 1:
                        continue
                    X += sum(dA[i][k][p - 1] * dB[j][k][q - 1] for k in range(K)) \
                        * 2 ** ((s + 1 - p - q) * b)
            w = math.ldexp(float(X), e[i] + f[j] - (s + 1) * b)
            v = alpha * w
            if beta != 0.0:
                v = float(Fraction(beta) * Fraction(C[i, j]) + Fraction(v))
            out[i, j] = v
    return out


@pytest.mark.parametrize("s,b,trim,phi", [(3, 7, 0, 0), (6, 7, 0, 8), (8, 7, 0, 0), (8, 7, 0, 32),
                                          (3, 8, 0, 0), (6, 8, 0, 8), (7, 8, 0, 32), (4, 8, 1, 0),
                                          (7, 8, 1, 8), (7, 8, 1, 32)])
def test_emul_gemm_bit_exact_against_rationals(orc, s, b, trim, phi):
    M, N, K = 4, 3, 9
    A, B, C = inputs.gemm_operands(90 + s + phi, M, N, K, kind="scaled", phi=phi)
    D, rc = orc.emul_gemm(1.5, A, B, 0.5, C, s, b=b, trim=trim)
    assert rc == 0
    ref = fraction_emul(1.5, A, B, 0.5, C, s, b, trim)
    assert np.array_equal(D, ref)


def test_int128_conversion_rounds_to_nearest_even(orc):
    vals = [0, 1, -1, 2 ** 53 + 1, 2 ** 53 + 3, -(2 ** 80) - 2 ** 27, 2 ** 100 + 2 ** 47,
            2 ** 100 + 2 ** 47 + 1, (1 << 126) - 1, -(1 << 127)]
    x = inputs.splitmix64(5, 0, 64)
    for i in range(0, 64, 2):
        v = (int(x[i]) << 64) | int(x[i + 1])
        vals.append(v >> int(x[i] % 60))
        vals.append(-(v >> int(x[i + 1] % 60)))
    for v in vals:
        assert orc.int128_to_double(v) == float(v), v


def test_emul_gemm_integer_inputs_bit_exact(orc):
    """Entries in {-8..8}: one 7-bit digit holds each exactly, so any s gives
    the exact integer product."""
    M, N, K = 12, 10, 64
    A, B, _ = inputs.gemm_operands(81, M, N, K, kind="int", with_c=False)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    for s in (3, 8):
        D, rc = orc.emul_gemm(1.0, A, B, 0.0, None, s)
        assert rc == 0 and np.array_equal(D, ref)


def test_emul_gemm_trim_special_cases(orc):
    """The trimmed last group changes nothing when it has no pair without a
    leading digit (s = 2) or when every entry fits one digit (integers in
    {-8..8}: all later digits are zero); otherwise it differs."""
    A, B, C = inputs.gemm_operands(87, 6, 5, 40, kind="scaled", phi=4)
    for b in (7, 8):
        full, _ = orc.emul_gemm(1.5, A, B, 0.5, C, 2, b=b)
        trimmed, _ = orc.emul_gemm(1.5, A, B, 0.5, C, 2, b=b, trim=True)
        assert np.array_equal(full, trimmed)
    Ai, Bi, _ = inputs.gemm_operands(81, 12, 10, 64, kind="int", with_c=False)
    ref = (Ai.astype(np.int64) @ Bi.astype(np.int64)).astype(np.float64)
    for s in (3, 7):
        D, rc = orc.emul_gemm(1.0, Ai, Bi, 0.0, None, s, b=8, trim=True)
        assert rc == 0 and np.array_equal(D, ref)
    full, _ = orc.emul_gemm(1.0, A, B, 0.0, None, 4, b=8)
    trimmed, _ = orc.emul_gemm(1.0, A, B, 0.0, None, 4, b=8, trim=True)
    assert not np.array_equal(full, trimmed)


def test_emul_gemm_special_cases(orc):
    M, N, K = 4, 3, 5
    A, B, C = inputs.gemm_operands(83, M, N, K)
    D, rc = orc.emul_gemm(0.0, np.full_like(A, np.nan), B, 0.5, C, 4)
    assert rc == 0 and np.array_equal(D, 0.5 * C)
    D, rc = orc.emul_gemm(1.0, A, B, 0.0, np.full_like(C, np.nan), 4)
    assert rc == 0 and not np.isnan(D).any()
    A2 = A.copy()
    A2[1, 1] = np.inf
    _, rc = orc.emul_gemm(1.0, A2, B, 0.0, None, 4)
    assert rc == 2
    Z = A.copy()
    Z[2] = 0.0                                          # zero row -> zero output row
    D, rc = orc.emul_gemm(1.0, Z, B, 0.0, None, 4)
    assert rc == 0 and np.all(D[2] == 0.0)


def test_emul_gemm_rows_match_full(orc):
    A, B, C = inputs.gemm_operands(85, 9, 7, 30, kind="scaled", phi=8)
    full, _ = orc.emul_gemm(1.5, A, B, 0.5, C, 6)
    part, _ = orc.emul_gemm(1.5, A, B, 0.5, C, 6, rows=np.array([8, 2]))
    assert np.array_equal(part, full[[8, 2]])


# ---- the FP32 variant of the emulated GEMM --------------------------------

U32 = 2.0 ** -24


def fraction_to_f32(x: Fraction) -> np.float32:
    """Nearest float32 to the rational x (ties to even, gradual underflow,
    overflow to infinity): the plain definition of one FP32 rounding."""
    if x == 0:
        return np.float32(0.0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)                       # below 2^-126: the subnormal spacing 2^-149
    unit = Fraction(2) ** (e - 23)
    q, r = divmod(a, unit)
    q = int(q)
    r = r / unit
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and q % 2 == 1):
        q += 1
    v = Fraction(q) * unit
    if v >= Fraction(2) ** 128:
        return np.float32(sign * np.inf)
    return np.float32(sign * float(v))       # q * unit has at most 25 bits: exact in double


def fraction_emul_f32(alpha, A, B, beta, C, s, b, trim=False):
    """The FP32 emulated GEMM in exact rationals: the digits and the integer X
    of fraction_emul, then (float)X, ldexpf, the float alpha product and the
    fused beta term, each rounded by fraction_to_f32."""
    M, K = A.shape
    N = B.shape[1]
    e = [math.frexp(float(np.max(np.abs(A[i]))))[1] if np.any(A[i]) else 0 for i in range(M)]
    f = [math.frexp(float(np.max(np.abs(B[:, j]))))[1] if np.any(B[:, j]) else 0
         for j in range(N)]
    dA = [[fraction_digits(float(A[i, k]), e[i], s, b) for k in range(K)] for i in range(M)]
    dB = [[fraction_digits(float(B[k, j]), f[j], s, b) for k in range(K)] for j in range(N)]
    out = np.empty((M, N), dtype=np.float32)
    for i in range(M):
        for j in range(N):
            X = 0
            for p in range(1, s + 1):
                for q in range(1, s + 2 - p):
                    if trim and p + q == s + 1 and min(p, q) > 1:
                        continue
                    X += sum(dA[i][k][p - 1] * dB[j][k][q - 1] for k in range(K)) \
                        * 2 ** ((s + 1 - p - q) * b)
            v = fraction_to_f32(Fraction(X))
            w = fraction_to_f32(Fraction(float(v)) * Fraction(2) ** (e[i] + f[j] - (s + 1) * b))
            o = fraction_to_f32(Fraction(float(np.float32(alpha))) * Fraction(float(w)))
            if beta != 0.0:
                o = fraction_to_f32(Fraction(float(np.float32(beta))) * Fraction(float(C[i, j]))
                                    + Fraction(float(o)))
            out[i, j] = o
    return out


def test_fraction_to_f32_matches_numpy_on_doubles():
    """The rounding helper against numpy's double -> float32 cast (one rounding
    when the source is a double), ties and subnormals included."""
    vals = [1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, -(1.0 + 2.0 ** -23 + 2.0 ** -24),
            2.0 ** -149, 2.0 ** -150, 3 * 2.0 ** -150, 2.0 ** -127 + 2.0 ** -150, 3.4e38, 3.5e38]
    rng = np.random.default_rng(5)
    vals += list(rng.standard_normal(200) * 2.0 ** rng.integers(-140, 120, 200))
    with np.errstate(over="ignore"):
        for v in vals:
            assert fraction_to_f32(Fraction(v)) == np.float32(v) or (
                np.isinf(np.float32(v)) and np.isinf(fraction_to_f32(Fraction(v)))), v


@pytest.mark.parametrize("s,b,trim,phi", [(2, 8, 0, 0), (3, 8, 0, 0), (3, 8, 0, 8), (3, 8, 1, 4),
                                          (4, 8, 0, 16), (3, 7, 0, 0), (4, 7, 0, 8)])
def test_emul_gemm_f32_bit_exact_against_rationals(orc, s, b, trim, phi):
    M, N, K = 4, 3, 9
    A, B, C = inputs.gemm_operands(190 + s + phi, M, N, K, kind="scaled", phi=phi)
    A, B, C = (x.astype(np.float32) for x in (A, B, C))
    D, rc = orc.emul_gemm_f32(1.5, A, B, 0.5, C, s, b=b, trim=trim)
    assert rc == 0 and D.dtype == np.float32
    ref = fraction_emul_f32(1.5, A, B, 0.5, C, s, b, trim)
    assert np.array_equal(D, ref)


@pytest.mark.parametrize("s,b", [(3, 8), (4, 7)])
def test_emul_gemm_f32_within_one_rounding_of_exact(orc, s, b):
    """With s b >= 24 + the exponent spread, the digits hold the FP32 inputs
    exactly and the kept pairs lose at most K 2^(-s b) of the scale, so the
    result is the exact product rounded once, up to that tiny term."""
    M, N, K = 6, 5, 40
    A, B, _ = inputs.gemm_operands(210 + s, M, N, K, kind="scaled", phi=0, with_c=False)
    A, B = A.astype(np.float32), B.astype(np.float32)
    D, _ = orc.emul_gemm_f32(1.0, A, B, 0.0, None, s, b=b)
    E = exact_gemm(1.0, A.astype(np.float64), B.astype(np.float64), 0.0, None)
    e, _ = orc.row_exponents(A.astype(np.float64))
    f, _ = orc.col_exponents(B.astype(np.float64))
    for i in range(M):
        for j in range(N):
            scale = Fraction(2) ** int(e[i] + f[j])
            tail = scale * K * Fraction(2) ** (-s * b) * (1 + Fraction(26, 100) * s)
            assert abs(Fraction(float(D[i, j])) - E[i][j]) <= \
                Fraction(U32 / 2) * abs(Fraction(float(D[i, j]))) + tail, (i, j)


def test_emul_gemm_f32_integer_and_special_cases(orc):
    Ai, Bi, _ = inputs.gemm_operands(81, 12, 10, 64, kind="int", with_c=False)
    ref = (Ai.astype(np.int64) @ Bi.astype(np.int64)).astype(np.float32)
    for s in (2, 3, 4):
        D, rc = orc.emul_gemm_f32(1.0, Ai, Bi, 0.0, None, s)
        assert rc == 0 and np.array_equal(D, ref)
    A, B, C = (x.astype(np.float32) for x in inputs.gemm_operands(83, 4, 3, 5))
    D, rc = orc.emul_gemm_f32(0.0, np.full_like(A, np.nan), B, 0.5, C, 3)
    assert rc == 0 and np.array_equal(D, np.float32(0.5) * C)
    D, rc = orc.emul_gemm_f32(1.0, A, B, 0.0, np.full_like(C, np.nan), 3)
    assert rc == 0 and not np.isnan(D).any()
    A2 = A.copy()
    A2[1, 1] = np.inf
    assert orc.emul_gemm_f32(1.0, A2, B, 0.0, None, 3)[1] == 2


# ---- the modular (CRT) variant of the emulated GEMM ------------------------

def fraction_crt(alpha, A, B, beta, C, k):
    """The CRT variant evaluated in exact rationals: k-bit integers by
    round-half-even of A 2^(k-e_i) and B 2^(k-f_j), their exact product, one
    rounding by Python's int -> float, math.ldexp, alpha in double, the fused
    beta term rounded once."""
    M, K = A.shape
    N = B.shape[1]
    e = [math.frexp(float(np.max(np.abs(A[i]))))[1] if np.any(A[i]) else 0 for i in range(M)]
    f = [math.frexp(float(np.max(np.abs(B[:, j]))))[1] if np.any(B[:, j]) else 0
         for j in range(N)]
    iA = [[round(Fraction(A[i, kk]) * Fraction(2) ** (k - e[i])) for kk in range(K)]
          for i in range(M)]
    iB = [[round(Fraction(B[kk, j]) * Fraction(2) ** (k - f[j])) for kk in range(K)]
          for j in range(N)]
    out = np.empty((M, N))
    for i in range(M):
        for j in range(N):
            P = sum(a * b for a, b in zip(iA[i], iB[j]))
            v = alpha * math.ldexp(float(P), e[i] + f[j] - 2 * k)
            if beta != 0.0:
                v = float(Fraction(beta) * Fraction(C[i, j]) + Fraction(v))
            out[i, j] = v
    return out


@pytest.mark.parametrize("k,phi", [(12, 0), (30, 4), (47, 0), (51, 8), (55, 32)])
def test_crt_gemm_bit_exact_against_rationals(orc, k, phi):
    M, N, K = 4, 3, 9
    A, B, C = inputs.gemm_operands(300 + k + phi, M, N, K, kind="scaled", phi=phi)
    A[0, 0] = 3 * 2.0 ** -60                              # far below the row's scale
    D, rc = orc.crt_gemm(1.5, A, B, 0.5, C, k)
    assert rc == 0
    assert np.array_equal(D, fraction_crt(1.5, A, B, 0.5, C, k))


@pytest.mark.parametrize("k", [40, 51])
def test_crt_gemm_within_derived_bound(orc, k):
    """|A' 2^(e-k) - A| <= 2^(e-k-1) entrywise, so the product differs from
    the exact one by at most sum_k (2^(e_i-k-1) |B_kj| + |A_ik| 2^(f_j-k-1) +
    2^(e_i+f_j-2k-2)), plus the final roundings."""
    M, N, K = 5, 4, 23
    A, B, C = inputs.gemm_operands(320 + k, M, N, K, kind="scaled", phi=8)
    D, _ = orc.crt_gemm(1.5, A, B, 0.5, C, k)
    E = exact_gemm(1.5, A, B, 0.5, C)
    e, _ = orc.row_exponents(A)
    f, _ = orc.col_exponents(B)
    for i in range(M):
        for j in range(N):
            t = sum(Fraction(2) ** int(e[i] - k - 1) * abs(Fraction(B[kk, j])) +
                    abs(Fraction(A[i, kk])) * Fraction(2) ** int(f[j] - k - 1) +
                    Fraction(2) ** int(e[i] + f[j] - 2 * k - 2) for kk in range(K))
            bud = Fraction(3) / Fraction(2) * t + Fraction(3 * U) * abs(Fraction(D[i, j])) + \
                Fraction(U) * abs(Fraction(0.5) * Fraction(C[i, j]))
            assert abs(Fraction(D[i, j]) - E[i][j]) <= bud, (i, j)


def test_crt_gemm_exact_cases(orc):
    """Integer entries in {-8..8} are k-bit integers exactly (k >= 4): the
    result is the exact product; rows sampling matches; zero rows stay zero;
    Inf is reported."""
    Ai, Bi, _ = inputs.gemm_operands(81, 12, 10, 64, kind="int", with_c=False)
    ref = (Ai.astype(np.int64) @ Bi.astype(np.int64)).astype(np.float64)
    for k in (4, 20, 51):
        D, rc = orc.crt_gemm(1.0, Ai, Bi, 0.0, None, k)
        assert rc == 0 and np.array_equal(D, ref)
    A, B, C = inputs.gemm_operands(85, 9, 7, 30, kind="scaled", phi=8)
    full, _ = orc.crt_gemm(1.5, A, B, 0.5, C, 51)
    part, _ = orc.crt_gemm(1.5, A, B, 0.5, C, 51, rows=np.array([8, 2]))
    assert np.array_equal(part, full[[8, 2]])
    Z = A.copy()
    Z[3] = 0.0
    D, _ = orc.crt_gemm(1.0, Z, B, 0.0, None, 51)
    assert np.all(D[3] == 0.0)
    Z[1, 1] = np.inf
    assert orc.crt_gemm(1.0, Z, B, 0.0, None, 51)[1] == 2
