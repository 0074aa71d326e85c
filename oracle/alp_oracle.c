/*
 * CPU oracle for the GEMM hot path.  TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the bench's CPU-baseline leg call it; the library never does.
 * It shares no code, header or table with the CUDA path.
 *
 * Everything here is written to be checked by eye against its definition:
 * plain loops, k ascending, no blocking, no reordering.
 *
 *   orc_gemm_f64      C = alpha*A*B + beta*C (Matthes et al. 2017, Eq. 1),
 *                     accumulated in long double, one final rounding to double.
 *   orc_absgemm       (|A||B|)_ij, the magnitude used by the error bound.
 *   orc_row_exponent  e_i of the emulated GEMM (frexp exponent of max_k |A_ik|).
 *   orc_split         digits of the emulated GEMM, in FP64 steps.
 *   orc_emul_gemm     the emulated FP64 GEMM end to end: exponents, digits,
 *                     exact integer slice products, FP64 recombination in its
 *                     fixed order.  The GPU must reproduce it bit for bit.
 *   orc_emul_gemm_f32 the same for FP32 operands and an FP32 result.
 *   orc_crt_gemm      the modular variant: the exact product of the operands
 *                     rounded to k-bit integers per row and column, rounded
 *                     once to FP64.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread (no fast-math, no
 * contraction, so every expression rounds exactly where it is written).
 */
#include <fenv.h>
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Row partitioning over host threads (rows are independent; no reductions). */

typedef void (*row_fn)(void* ctx, int64_t r);

typedef struct {
    row_fn fn;
    void* ctx;
    int64_t r0, r1;
} span_t;

static void* span_run(void* p) {
    span_t* s = (span_t*)p;
    for (int64_t r = s->r0; r < s->r1; ++r) s->fn(s->ctx, r);
    return NULL;
}

static void for_rows(int64_t nrows, int nthreads, row_fn fn, void* ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > nrows) nthreads = (int)(nrows > 0 ? nrows : 1);
    if (nthreads == 1) {
        for (int64_t r = 0; r < nrows; ++r) fn(ctx, r);
        return;
    }
    pthread_t tid[256];
    span_t sp[256];
    for (int t = 0; t < nthreads; ++t) {
        sp[t].fn = fn;
        sp[t].ctx = ctx;
        sp[t].r0 = nrows * t / nthreads;
        sp[t].r1 = nrows * (t + 1) / nthreads;
        pthread_create(&tid[t], NULL, span_run, &sp[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(tid[t], NULL);
}

/* ------------------------------------------------------------------------- */
/* O1: the plain definition of the GEMM, Eq. 1 of Matthes et al. 2017,       */
/* generalised to M x K times K x N, row-major with leading dimensions.      */

typedef struct {
    int64_t M, N, K;
    double alpha, beta;
    const double *A, *B, *C;
    int64_t lda, ldb, ldc;
    double* D;
    int64_t ldd;
    const int64_t* rows;
    int absval;
} gemm_ctx;

static void gemm_row(void* p, int64_t r) {
    gemm_ctx* g = (gemm_ctx*)p;
    int64_t i = g->rows ? g->rows[r] : r;
    double* d = g->D + r * g->ldd;
    for (int64_t j = 0; j < g->N; ++j) {
        if (g->absval) {
            long double s = 0.0L;
            for (int64_t k = 0; k < g->K; ++k)
                s += fabsl((long double)g->A[i * g->lda + k]) * fabsl((long double)g->B[k * g->ldb + j]);
            d[j] = (double)s;
            continue;
        }
        /* BLAS convention: alpha == 0 or K == 0 forms no product and reads
         * neither A nor B; beta == 0 reads no C. */
        if (g->alpha == 0.0 || g->K == 0) {
            d[j] = (g->beta == 0.0) ? 0.0 : g->beta * g->C[i * g->ldc + j];
            continue;
        }
        long double s = 0.0L;
        for (int64_t k = 0; k < g->K; ++k)
            s += (long double)g->A[i * g->lda + k] * (long double)g->B[k * g->ldb + j];
        long double v = (long double)g->alpha * s;
        if (g->beta != 0.0) v += (long double)g->beta * (long double)g->C[i * g->ldc + j];
        d[j] = (double)v;
    }
}

/* D[r, :] = alpha * A[i, :] B + beta * C[i, :] for i = rows[r] (or i = r when
 * rows == NULL, nrows == M).  D may equal C only when rows == NULL and
 * ldd == ldc (each row is read before it is written). */
int orc_gemm_f64(int64_t M, int64_t N, int64_t K, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb,
                 double beta, const double* C, int64_t ldc,
                 double* D, int64_t ldd, const int64_t* rows, int64_t nrows, int nthreads) {
    if (M < 0 || N < 0 || K < 0) return 1;
    gemm_ctx g = {M, N, K, alpha, beta, A, B, C, lda, ldb, ldc, D, ldd, rows, 0};
    for_rows(rows ? nrows : M, nthreads, gemm_row, &g);
    return 0;
}

/* D[r, j] = sum_k |A_ik| |B_kj| (long double, rounded once). */
int orc_absgemm(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                const double* B, int64_t ldb, double* D, int64_t ldd,
                const int64_t* rows, int64_t nrows, int nthreads) {
    if (M < 0 || N < 0 || K < 0) return 1;
    gemm_ctx g = {M, N, K, 1.0, 0.0, A, B, NULL, lda, ldb, 0, D, ldd, rows, 1};
    for_rows(rows ? nrows : M, nthreads, gemm_row, &g);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* O2: the emulated FP64 GEMM (error-free splitting after Ozaki, Ogita, Oishi */
/* and Rump, Numer. Algorithms 59, 2012), in the reading this library uses:  */
/*                                                                           */
/*  scale    e_i = exponent of max_k |A_ik| as returned by frexp, so that    */
/*           every r0_ik = A_ik * 2^-e_i lies in (-1, 1); e_i = 0 for a zero */
/*           row.  f_j likewise for the columns of B.                        */
/*  digits   for p = 1..s:  x = r_{p-1} * 2^b,  d_p = nearest integer to x   */
/*           (ties to even),  r_p = x - d_p.  All steps are exact in FP64.   */
/*  products S^t = sum_{p+q=t} D_A^p (D_B^q)^T, t = 2..s+1, exact integers.  */
/*           Trimmed variant (trim = 1): the last group t = s+1 keeps only   */
/*           the pairs with a leading digit, (1, s) and (s, 1).              */
/*  combine  X = sum_t S^t 2^((s+1-t) b)  exactly (an integer below 2^100),  */
/*           v = X rounded once to the nearest double (ties to even),        */
/*           w = v * 2^(e_i + f_j - (s+1) b)  (one rounding if subnormal),   */
/*           out = alpha*w, then fma(beta, C_ij, out) when beta != 0.        */
/*  So the FP64 result is the correctly rounded value of the kept digit      */
/*  products; the only error besides the last three roundings is the digits */
/*  that were cut off.                                                       */

/* Exponent of max_k |X[i, k]| (frexp convention).  Returns 1 if an Inf or
 * NaN is present, else 0. */
int orc_row_exponents(int64_t M, int64_t K, const double* X, int64_t ldx, int32_t* e) {
    int bad = 0;
    for (int64_t i = 0; i < M; ++i) {
        double m = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            double a = X[i * ldx + k];
            if (!isfinite(a)) bad = 1;
            else if (fabs(a) > m) m = fabs(a);
        }
        int ex = 0;
        if (m != 0.0) frexp(m, &ex);
        e[i] = ex;
    }
    return bad;
}

/* Column version for row-major B (K x N): f_j from max_k |B[k, j]|. */
int orc_col_exponents(int64_t K, int64_t N, const double* X, int64_t ldx, int32_t* f) {
    int bad = 0;
    for (int64_t j = 0; j < N; ++j) {
        double m = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            double a = X[k * ldx + j];
            if (!isfinite(a)) bad = 1;
            else if (fabs(a) > m) m = fabs(a);
        }
        int ex = 0;
        if (m != 0.0) frexp(m, &ex);
        f[j] = ex;
    }
    return bad;
}

/* Digits of one value: r0 = x * 2^-e, then s steps of b bits. */
static void split_value(double x, int32_t e, int s, int b, int32_t* d, double* rem) {
    double r = ldexp(x, -e);
    for (int p = 0; p < s; ++p) {
        double y = ldexp(r, b);
        double q = nearbyint(y);     /* round-to-nearest-even in the default mode */
        d[p] = (int32_t)q;
        r = y - q;
    }
    if (rem) *rem = r;
}

/* Digits of a row-major R x K matrix with one exponent per row.
 * Out: digit[p][i][k] as int32 (p = 0..s-1 holds digit p+1), rem[i][k] the
 * final remainder r_s (may be NULL). */
int orc_split(int64_t R, int64_t K, const double* X, int64_t ldx, const int32_t* e,
              int s, int b, int32_t* digit, double* rem) {
    int32_t d[16];
    if (s < 1 || s > 16) return 1;
    if (fegetround() != FE_TONEAREST) return 1;
    for (int64_t i = 0; i < R; ++i)
        for (int64_t k = 0; k < K; ++k) {
            double rr;
            split_value(X[i * ldx + k], e[i], s, b, d, &rr);
            for (int p = 0; p < s; ++p) digit[((int64_t)p * R + i) * K + k] = d[p];
            if (rem) rem[i * K + k] = rr;
        }
    return 0;
}

typedef struct {
    int64_t M, N, K;
    double alpha, beta;
    const double* C;
    int64_t ldc;
    double* D;
    int64_t ldd;
    const int64_t* rows;
    int s, b, trim;
    const int16_t *dA, *dB;   /* [s][nrows][K] (row r of the output), [s][N][K] */
    int64_t nra;
    const int32_t *e, *f;
    int out_f32;              /* FP32 result: float rounding, float alpha and beta */
} emul_ctx;

static void emul_row(void* p, int64_t r) {
    emul_ctx* g = (emul_ctx*)p;
    int64_t i = g->rows ? g->rows[r] : r;
    double* d = g->D + r * g->ldd;
    const int s = g->s, b = g->b;
    for (int64_t j = 0; j < g->N; ++j) {
        if (g->alpha == 0.0 || g->K == 0) {
            if (g->out_f32)
                d[j] = (g->beta == 0.0) ? 0.0 : (double)((float)g->beta * (float)g->C[i * g->ldc + j]);
            else
                d[j] = (g->beta == 0.0) ? 0.0 : g->beta * g->C[i * g->ldc + j];
            continue;
        }
        __int128 X = 0;                                     /* exact */
        for (int t = 2; t <= s + 1; ++t) {
            int64_t S = 0;
            for (int pa = 1; pa <= s; ++pa) {
                int qb = t - pa;
                if (qb < 1 || qb > s) continue;
                if (g->trim && t == s + 1 && pa != 1 && qb != 1) continue;
                const int16_t* a = g->dA + ((int64_t)(pa - 1) * g->nra + r) * g->K;
                const int16_t* bb = g->dB + ((int64_t)(qb - 1) * g->N + j) * g->K;
                for (int64_t k = 0; k < g->K; ++k) S += (int64_t)a[k] * (int64_t)bb[k];
            }
            X += (__int128)S * ((__int128)1 << ((s + 1 - t) * b));
        }
        if (g->out_f32) {
            /* |X| < 2^63 for s * b <= 32: (float) of the int64 rounds once */
            float v = ldexpf((float)(int64_t)X, g->e[i] + g->f[j] - (s + 1) * b);
            float out = (float)g->alpha * v;
            if (g->beta != 0.0) out = fmaf((float)g->beta, (float)g->C[i * g->ldc + j], out);
            d[j] = (double)out;
            continue;
        }
        double v = ldexp((double)X, g->e[i] + g->f[j] - (s + 1) * b);   /* (double) rounds once */
        double out = g->alpha * v;
        if (g->beta != 0.0) out = fma(g->beta, g->C[i * g->ldc + j], out);
        d[j] = out;
    }
}

typedef struct {
    const double* X;
    int64_t K, ldx;
    const int32_t* e;
    const int64_t* rows;
    int s, b;
    int16_t* out;     /* [s][nrows][K] */
    int64_t nrows;
} split_ctx;

static void split_row(void* p, int64_t r) {
    split_ctx* c = (split_ctx*)p;
    const int64_t i = c->rows ? c->rows[r] : r;
    int32_t d[16];
    for (int64_t k = 0; k < c->K; ++k) {
        split_value(c->X[i * c->ldx + k], c->e[i], c->s, c->b, d, NULL);
        for (int q = 0; q < c->s; ++q) c->out[((int64_t)q * c->nrows + r) * c->K + k] = (int16_t)d[q];
    }
}

static int emul_gemm(int64_t M, int64_t N, int64_t K, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb,
                     double beta, const double* C, int64_t ldc,
                     double* D, int64_t ldd, int s, int b, int trim,
                     const int64_t* rows, int64_t nrows, int nthreads, int out_f32) {
    const int64_t nra = rows ? nrows : M;
    int32_t* e = (int32_t*)calloc((size_t)(M > 0 ? M : 1), sizeof(int32_t));
    int32_t* f = (int32_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(int32_t));
    int bad = orc_row_exponents(M, K, A, lda, e) | orc_col_exponents(K, N, B, ldb, f);
    if (bad && alpha != 0.0) { free(e); free(f); return 2; }
    size_t na = (size_t)s * (size_t)nra * (size_t)K, nb = (size_t)s * (size_t)N * (size_t)K;
    int16_t* dA = (int16_t*)malloc((na ? na : 1) * sizeof(int16_t));
    int16_t* dB = (int16_t*)malloc((nb ? nb : 1) * sizeof(int16_t));
    size_t nt = (size_t)N * (size_t)K;
    double* Bt = (double*)malloc((nt ? nt : 1) * sizeof(double));
    for (int64_t k = 0; k < K; ++k)
        for (int64_t j = 0; j < N; ++j) Bt[j * K + k] = B[k * ldb + j];
    split_ctx sa = {A, K, lda, e, rows, s, b, dA, nra};
    for_rows(nra, nthreads, split_row, &sa);
    split_ctx sb = {Bt, K, K, f, NULL, s, b, dB, N};
    for_rows(N, nthreads, split_row, &sb);
    emul_ctx g = {M, N, K, alpha, beta, C, ldc, D, ldd, rows, s, b, trim, dA, dB, nra, e, f,
                  out_f32};
    for_rows(nra, nthreads, emul_row, &g);
    free(Bt); free(dA); free(dB); free(e); free(f);
    return 0;
}

/* Emulated GEMM with s digits of b bits (s*b + 32 < 127 keeps X in range);
 * trim = 1 selects the trimmed last group.  Returns 0, or 2 when A or B holds
 * an Inf or NaN (the emulated path does not support them), 1 on bad sizes. */
int orc_emul_gemm(int64_t M, int64_t N, int64_t K, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb,
                  double beta, const double* C, int64_t ldc,
                  double* D, int64_t ldd, int s, int b, int trim,
                  const int64_t* rows, int64_t nrows, int nthreads) {
    if (M < 0 || N < 0 || K < 0 || s < 1 || s > 16 || b < 1 || b > 15 || s * b > 90 ||
        (trim != 0 && trim != 1))
        return 1;
    return emul_gemm(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s, b, trim, rows,
                     nrows, nthreads, 0);
}

/* The same for FP32 operands (A, B, C, alpha and beta hold float values,
 * passed as double, which is exact): the digits and the exact integer sum X
 * are those above; the result is v = ldexpf((float)X, e_i + f_j - (s+1) b)
 * (one rounding, a second only when v is subnormal), out = (float)alpha * v,
 * then fmaf((float)beta, C_ij, out) when beta != 0, all in float arithmetic.
 * s * b <= 32 keeps |X| below 2^63.  D receives the float results. */
int orc_emul_gemm_f32(int64_t M, int64_t N, int64_t K, double alpha,
                      const double* A, int64_t lda, const double* B, int64_t ldb,
                      double beta, const double* C, int64_t ldc,
                      double* D, int64_t ldd, int s, int b, int trim,
                      const int64_t* rows, int64_t nrows, int nthreads) {
    if (M < 0 || N < 0 || K < 0 || s < 1 || b < 1 || s * b > 32 || (trim != 0 && trim != 1))
        return 1;
    return emul_gemm(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s, b, trim, rows,
                     nrows, nthreads, 1);
}

/* ------------------------------------------------------------------------- */
/* O2b: the modular (CRT) variant of the emulated FP64 GEMM, after Ozaki,    */
/* Uchino and Imamura's scheme II, in the reading this library uses: with    */
/* the row and column exponents e_i, f_j of O2,                              */
/*   A'_ik = nearest integer (ties to even) to A_ik 2^(k - e_i),             */
/*   B'_kj = nearest integer (ties to even) to B_kj 2^(k - f_j),             */
/*   P_ij  = sum_k A'_ik B'_kj   (exact),                                    */
/*   out   = alpha * ldexp((double)P_ij, e_i + f_j - 2k)  (one rounding;     */
/*           a second only when subnormal), then fma(beta, C_ij, out).       */
/* The GPU computes P from its residues modulo pairwise coprime moduli and   */
/* the Chinese remainder theorem; this is the plain definition it must meet  */
/* bit for bit.  |A'| <= 2^k, so |P| <= K 2^(2k); the caller keeps that      */
/* below 2^125.                                                              */

typedef struct {
    int64_t M, N, K;
    double alpha, beta;
    const double* C;
    int64_t ldc;
    double* D;
    int64_t ldd;
    const int64_t* rows;
    int k;
    const int64_t *iA, *iB;   /* [nrows][K] scaled rows of A, [N][K] scaled columns of B */
    const int32_t *e, *f;
} crt_ctx;

static void crt_row(void* p, int64_t r) {
    crt_ctx* g = (crt_ctx*)p;
    const int64_t i = g->rows ? g->rows[r] : r;
    double* d = g->D + r * g->ldd;
    for (int64_t j = 0; j < g->N; ++j) {
        if (g->alpha == 0.0 || g->K == 0) {
            d[j] = (g->beta == 0.0) ? 0.0 : g->beta * g->C[i * g->ldc + j];
            continue;
        }
        __int128 P = 0;
        const int64_t* a = g->iA + r * g->K;
        const int64_t* b = g->iB + j * g->K;
        for (int64_t kk = 0; kk < g->K; ++kk) P += (__int128)a[kk] * (__int128)b[kk];
        double v = ldexp((double)P, g->e[i] + g->f[j] - 2 * g->k);
        double out = g->alpha * v;
        if (g->beta != 0.0) out = fma(g->beta, g->C[i * g->ldc + j], out);
        d[j] = out;
    }
}

/* Nearest integer (ties to even) to x 2^(k - e): ldexp is exact unless the
 * result is below the normal range, where the nearest integer is 0 anyway. */
static int64_t scaled_int(double x, int32_t e, int k) {
    return (int64_t)nearbyint(ldexp(x, k - e));
}

int orc_crt_gemm(int64_t M, int64_t N, int64_t K, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb,
                 double beta, const double* C, int64_t ldc,
                 double* D, int64_t ldd, int k,
                 const int64_t* rows, int64_t nrows, int nthreads) {
    if (M < 0 || N < 0 || K < 0 || k < 1 || k > 60) return 1;
    if (K > 0 && (int)(2 * k) + (int)ceil(log2((double)K)) > 125) return 1;
    const int64_t nra = rows ? nrows : M;
    int32_t* e = (int32_t*)calloc((size_t)(M > 0 ? M : 1), sizeof(int32_t));
    int32_t* f = (int32_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(int32_t));
    int bad = orc_row_exponents(M, K, A, lda, e) | orc_col_exponents(K, N, B, ldb, f);
    if (bad && alpha != 0.0) { free(e); free(f); return 2; }
    size_t na = (size_t)nra * (size_t)K, nb = (size_t)N * (size_t)K;
    int64_t* iA = (int64_t*)malloc((na ? na : 1) * sizeof(int64_t));
    int64_t* iB = (int64_t*)malloc((nb ? nb : 1) * sizeof(int64_t));
    for (int64_t r = 0; r < nra; ++r) {
        const int64_t i = rows ? rows[r] : r;
        for (int64_t kk = 0; kk < K; ++kk) iA[r * K + kk] = scaled_int(A[i * lda + kk], e[i], k);
    }
    for (int64_t j = 0; j < N; ++j)
        for (int64_t kk = 0; kk < K; ++kk) iB[j * K + kk] = scaled_int(B[kk * ldb + j], f[j], k);
    crt_ctx g = {M, N, K, alpha, beta, C, ldc, D, ldd, rows, k, iA, iB, e, f};
    for_rows(nra, nthreads, crt_row, &g);
    free(iA); free(iB); free(e); free(f);
    return 0;
}

/* Significand bits of long double on this host (64 on x86_64, 113 on aarch64),
 * for the tests' error budget. */
int orc_long_double_digits(void) { return LDBL_MANT_DIG; }

/* Nearest double of a 128-bit integer given as hi*2^64 + lo (two's
 * complement), for the tests' check of the conversion above. */
double orc_int128_to_double(int64_t hi, uint64_t lo) {
    __int128 x = ((__int128)hi << 64) | (__int128)lo;
    return (double)x;
}
