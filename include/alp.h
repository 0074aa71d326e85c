/*
 * alp.h -- C-ABI of the GB300 (sm_103a) double-precision GEMM library.
 *
 * The operation is the general matrix multiplication of Matthes, Widera,
 * Zenker, Worpitz, Huebl and Bussmann, "Tuning and optimization for a variety
 * of many-core architectures without changing a single line of implementation
 * code using the Alpaka library" (P^3MA 2017), Eq. 1:
 *
 *        C = alpha * A * B + beta * C
 *
 * generalised from the paper's square N x N matrices (Sect. 2) to
 *   A: M x K, row-major, leading dimension lda >= K   (element (i,k) at A[i*lda+k])
 *   B: K x N, row-major, leading dimension ldb >= N   (element (k,j) at B[k*ldb+j])
 *   C: M x N, row-major, leading dimension ldc >= N   (element (i,j) at C[i*ldc+j])
 * all IEEE binary64.  The tile parameters the paper tunes (tile size T and the
 * per-thread element block, Sect. 2.1, Listing 1, Table 4) are the fields of
 * alp_config below.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers: A, B, C, workspaces and the batched pointer/size arrays are DEVICE
 *   pointers owned by the caller; the library never frees them.  "h"-prefixed
 *   arrays and alp_config / out-parameters are HOST pointers.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  GEMM calls are asynchronous and enqueue work only on `stream`;
 *   the one exception is the modular scheme with nslices = 0, which waits for
 *   its operand statistics once (alp_emul_crt_choose).
 * BLAS semantics (the paper does not say): beta == 0 reads no C (NaN in C does
 *   not propagate); alpha == 0 or K == 0 reads neither A nor B and sets
 *   C = beta*C; M == 0 or N == 0 returns ALP_OK without launching anything.
 *   A and B must not overlap C.
 * Errors: argument errors are returned synchronously before anything is
 *   launched.  Faults found by a kernel (an operand with Inf/NaN on the
 *   emulated path, a wait that timed out) are recorded in a device error word
 *   that alp_get_device_error() reads and clears; no C++ exception crosses the
 *   ABI and no kernel traps.
 */
#ifndef ALP_H
#define ALP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum alp_status {
    ALP_OK = 0,
    ALP_ERR_INVALID_ARG = 1,   /* bad size, leading dimension, pointer or config */
    ALP_ERR_UNSUPPORTED = 2,   /* valid request this build cannot do (see each call) */
    ALP_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    ALP_ERR_TIMEOUT = 4,       /* a device-side wait ran past its limit */
    ALP_ERR_WORKSPACE = 5,     /* workspace NULL or smaller than the *_workspace query */
    ALP_ERR_NOT_TUNED = 6      /* PREDICT asked for but no trained cost model loaded */
} alp_status;

typedef enum alp_slice_kind {
    ALP_SLICE_INT8 = 0,        /* not available on sm_103a: tcgen05 has no kind::i8 there */
    ALP_SLICE_BF16 = 1,        /* digits of 7 bits held exactly in bf16; 3..8 slices, K <= 32768 */
    ALP_SLICE_BF16_B8 = 2,     /* digits of 8 bits held exactly in bf16; 3..7 slices, K <= 14336 */
    ALP_SLICE_BF16_B8_TRIM = 3, /* as ALP_SLICE_BF16_B8, but the last group t = nslices+1 keeps
                                  only the pairs with a leading digit, (1, s) and (s, 1) */
    ALP_SLICE_BF16_CRT = 4     /* modular scheme: residues modulo nslices (4..16) pairwise
                                  coprime moduli, one product per modulus (see below) */
} alp_slice_kind;

typedef enum alp_path { ALP_PATH_NATIVE = 0, ALP_PATH_EMUL = 1 } alp_path;

typedef enum alp_tune_mode {
    ALP_TUNE_EXHAUSTIVE = 0,   /* time every valid config on the GPU, keep the fastest */
    ALP_TUNE_PREDICT = 1,      /* argmin of the loaded cost model over valid configs */
    ALP_TUNE_LOOKUP = 2        /* tuned-config cache only (ALP_ERR_NOT_TUNED if absent) */
} alp_tune_mode;

/*
 * Tile configuration of the native kernel (the paper's tuning knobs, Sect. 2.1
 * and Table 4, on a GPU re-read as one C tile per thread block):
 *   bm, bn  C tile of one thread block, in {64, 128, 256}
 *   bk      K step of one pipeline stage, in {16, 32, 64}
 *   tm, tn  per-thread register tile (the element layer), in {2, 4, 8};
 *           a warp covers (8*tm) x (4*tn) of C, the block (bm/tm)*(bn/tn) threads
 *   stages  depth of the shared-memory ring; 0 = as many as fit (at most 4)
 * Its shared memory per stage is (bm + bn) * bk * 8 bytes, the block version of
 * the tile cache model K(S,T) = 2 T^2 S of Eq. 3.
 */
typedef struct alp_config {
    int32_t bm, bn, bk, tm, tn, stages;
} alp_config;

/* Human-readable name of a status code (static storage). */
const char* alp_status_string(alp_status s);

/*
 * Native FP64 GEMM, Eq. 1 (Sect. 2, Fig. 2): TMA-staged A and B tiles in a
 * multi-stage mbarrier ring, FP64 DMMA tensor-core MMAs into per-thread
 * register tiles, alpha/beta epilogue.  cfg == NULL selects the config from the
 * tuned cache, else the loaded cost model, else the built-in default.
 * Operands whose base address is not 16-byte aligned, or whose lda/ldb is odd,
 * run through a non-TMA variant of the same kernel.
 * Returns ALP_ERR_INVALID_ARG for negative sizes, ld < row width, NULL
 * operands that would be read, or an invalid cfg.
 */
alp_status alp_gemm_f64(int64_t M, int64_t N, int64_t K, double alpha,
                        const double* A, int64_t lda, const double* B, int64_t ldb,
                        double beta, double* C, int64_t ldc,
                        const alp_config* cfg, void* stream);
/* Transposed operands for the native GEMM: C = alpha op(A) op(B) + beta C with
 * op(X) = X (trans 0) or X^T (trans 1), storage as for alp_gemm_f64_emul_ex.
 * A transposed operand is first packed row-major into `workspace` (one read
 * and one write of it, small against the 2 M N K FP64 flops), then the product
 * runs as alp_gemm_f64 with `cfg`; results are bit-identical to alp_gemm_f64
 * on the transposed matrices.  workspace >= alp_gemm_f64_ex_workspace(...),
 * 256-byte aligned (none needed, and none read, when neither is transposed). */
alp_status alp_gemm_f64_ex(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                           double alpha, const double* A, int64_t lda, const double* B,
                           int64_t ldb, double beta, double* C, int64_t ldc,
                           const alp_config* cfg, void* workspace, size_t workspace_bytes,
                           void* stream);
size_t alp_gemm_f64_ex_workspace(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K);

/*
 * Emulated FP64 GEMM (not in the paper; error-free splitting after Ozaki,
 * Ogita, Oishi and Rump 2012).  Per row i of A, e_i = frexp exponent of
 * max_k |A_ik|; every A_ik * 2^-e_i is cut into `nslices` digits of b bits
 * (b = 7 for ALP_SLICE_BF16, 8 for ALP_SLICE_BF16_B8; round to nearest even,
 * held exactly in bf16); likewise the columns of B with exponents f_j.  The
 * slice products S^t = sum_{p+q=t} D_A^p (D_B^q)^T, t = 2..nslices+1 (for
 * ALP_SLICE_BF16_B8_TRIM, S^(nslices+1) sums only the pairs (1, nslices) and
 * (nslices, 1): s(s-1)/2 + 2 products instead of s(s+1)/2), run on
 * tcgen05 tensor cores with exact integer-valued fp32 partial sums (drained
 * every 2^(22-2b)..2^(24-2b) k into int32), and are recombined exactly and
 * rounded once to FP64:
 *   X = sum_t S^t 2^(b(nslices+1-t)),  C = alpha * (X rounded to nearest,
 *   times 2^(e_i + f_j - b(nslices+1)))  (+ fma(beta, C, .) when beta != 0).
 * nslices in 3..8 (b = 7) or 3..7 (b = 8, either kind).  ALP_SLICE_INT8 returns
 * ALP_ERR_UNSUPPORTED on sm_103a, whose tcgen05 has no kind::i8.
 * K <= 32768 (b = 7) or 14336 (b = 8) (int32 group sums; larger K returns
 * ALP_ERR_UNSUPPORTED).
 * Inf/NaN in A or B is reported as ALP_ERR_UNSUPPORTED through
 * alp_get_device_error() and C is left unspecified.  workspace: device memory
 * of at least alp_gemm_f64_emul_workspace(...) bytes, 256-byte aligned, owned
 * by the caller, not read by the caller afterwards.
 */
alp_status alp_gemm_f64_emul(int64_t M, int64_t N, int64_t K, double alpha,
                             const double* A, int64_t lda, const double* B, int64_t ldb,
                             double beta, double* C, int64_t ldc, int nslices,
                             alp_slice_kind kind, void* workspace, size_t workspace_bytes,
                             void* stream);

/* Bytes of workspace alp_gemm_f64_emul needs (0 for invalid arguments). */
size_t alp_gemm_f64_emul_workspace(int64_t M, int64_t N, int64_t K, int nslices,
                                   alp_slice_kind kind);

/*
 * Stages of the emulated GEMM, exposed for testing and per-stage timing (the
 * same kernels alp_gemm_f64_emul launches, in this order).
 * alp_emul_exponents: e[i] (int32, device) for the `rows` rows of a row-major
 * rows x cols X (trans == 0), or f[j] for the `rows` columns of a row-major
 * cols x rows X (trans == 1).  alp_emul_split: digits of a
 * row-major R x K matrix given its per-row exponents, written as bf16 to
 * out[p][r][k] (p = 0..nslices-1, row stride kpad elements, kpad >= K, zero
 * filled beyond K); for a K x N row-major B pass trans = 1, R = N and the
 * result is the transposed digit matrix out[p][n][k].  kind fixes b (7 for
 * ALP_SLICE_BF16, 8 for the other two); every stage of one product takes the
 * same kind.
 */
alp_status alp_emul_exponents(int64_t rows, int64_t cols, const double* X, int64_t ldx,
                              int trans, int32_t* exps, void* stream);
alp_status alp_emul_split(int64_t R, int64_t K, const double* X, int64_t ldx, int trans,
                          const int32_t* exps, int nslices, alp_slice_kind kind, void* out_bf16,
                          int64_t kpad, void* stream);
/* The modular kinds only: alp_emul_exponents (trans = 0) and alp_emul_split
 * (trans = 0) of the same rows in one kernel, which reads each row twice (the
 * second time from L2) instead of scanning the matrix in a launch of its own;
 * exps receives the row exponents.  The same results as the two calls bit for
 * bit.  out_bf16 8-byte aligned, kpad a multiple of 64 and >= K, ldx >= K;
 * alp_gemm_f64_emul uses it for A when nslices > 0 and A is not transposed.
 * ALP_ERR_INVALID_ARG for other kinds. */
alp_status alp_emul_scan_split_rows(int64_t R, int64_t K, const double* X, int64_t ldx,
                                    int32_t* exps, int nslices, alp_slice_kind kind,
                                    void* out_bf16, int64_t kpad, void* stream);
/* alp_emul_slice_products: the tensor-core stage, S^t = sum_{p+q=t}
 * D_A^p (D_B^q)^T for t = 2..nslices+1 as exact int32 into
 * G[t-2][m][n] (row stride ldg, ldg a multiple of 256 and >= N; plane stride
 * M*ldg), from digit slices da[p][m][k] (M x kpad) and db[p][n][k] (N x kpad)
 * as written by alp_emul_split with the same kind (ALP_SLICE_BF16_B8_TRIM:
 * the last group sums only its two leading-digit pairs); kpad a multiple of
 * 64, K <= 32768 (b = 7) or 14336 (b = 8) (65472 for the modular kind).
 * alp_emul_recombine: C = alpha * round(sum_t S^t 2^(b(nslices+1-t))) *
 * 2^(e_i + f_j - b(nslices+1)) (+ fma(beta, C, .)) from those sums.
 * G is 16-byte aligned.  For the modular kind (below) G holds bytes, not
 * int32: plane l (stride M*ldg bytes) holds x_l = (P y_l) mod m_{l+1}. */
alp_status alp_emul_slice_products(int64_t M, int64_t N, int64_t K, int nslices,
                                   alp_slice_kind kind, const void* da_bf16, const void* db_bf16,
                                   int64_t kpad, void* G, int64_t ldg, void* stream);
alp_status alp_emul_recombine(int64_t M, int64_t N, int nslices, alp_slice_kind kind,
                              const int32_t* G, int64_t ldg, const int32_t* e, const int32_t* f,
                              double alpha, double beta, double* C, int64_t ldc, void* stream);

/*
 * The modular scheme, ALP_SLICE_BF16_CRT (not in the paper; after Ozaki,
 * Uchino and Imamura's scheme II, 2024).  With n = nslices moduli m_1..m_n,
 * the first n of 256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217,
 * 211, 199, 197, 193 (pairwise coprime, product Mn), and
 * k = alp_emul_crt_bits(K, n), the largest k <= 60 with
 * K 2^(2k+1) <= Mn (1 - 2^-18):
 *   A'_ik = RN(A_ik 2^(k - e_i)), B'_kj = RN(B_kj 2^(k - f_j)) (integers,
 *   |.| <= 2^k, e_i and f_j the exponents above),
 *   P = A' B' exact (|P| <= K 2^(2k) < Mn / 2),
 *   C = alpha * RN(P 2^(e_i + f_j - 2k))  (+ fma(beta, C, .) when beta != 0).
 * P is reached through its residues: the split writes out[l][r][k] = a residue
 * of A'_rk modulo m_{l+1} of magnitude at most 128 (exact in bf16; the one
 * nearest to zero, or, for k <= 51, one modulus off it when A'/m lies within
 * 0.003 of a half-integer); the tensor-core stage sums
 * Q_l = sum_k a_l b_l exactly (|Q_l| <= K 2^14, Q_l = P mod m_l) and writes
 * the byte x_l = (Q_l y_l) mod m_l, y_l = (Mn/m_l)^-1 mod m_l, into plane
 * l-1 of G; the recombination forms sum_l x_l (Mn/m_l) = P mod Mn in 128-bit
 * integers (the Chinese remainder theorem) and rounds once.  n products of
 * K digits instead of the digit scheme's s(s+1)/2.
 * n in 4..16, or n = 0 for an automatic count (below), K <= 65472 (1023
 * blocks of 64; |Q_l| <= K 2^14 < 2^30); FP64 only (the FP32 calls return
 * ALP_ERR_UNSUPPORTED for this kind).  The error comes from the two operand
 * roundings, at most 2^(e_i-k-1) per entry of A (2^(f_j-k-1) of B): for
 * K = 8192 and entries of one magnitude, 14 moduli (k = 48) stay below the
 * native kernel's error and 15 (k = 51) well below; entries spread over
 * 2^(+-8) need 15, over 2^(+-32) 16.  With nslices = 0, alp_gemm_f64_emul and
 * alp_gemm_f64_emul_ex choose n as alp_emul_crt_choose does: this
 * synchronises `stream` once (the statistics are read back) and needs
 * alp_gemm_f64_emul_workspace(M, N, K, 0, ALP_SLICE_BF16_CRT) bytes (the
 * 16-moduli layout).  alp_gemm_f64_emul, alp_gemm_f64_emul_ex, the workspace
 * query, alp_emul_split and alp_emul_slice_products accept the kind;
 * alp_emul_recombine does not (it has no K): use alp_emul_recombine_crt,
 * which reads the n byte planes R[l][i][j] = (P_ij y_{l+1}) mod m_{l+1}
 * (row stride ldr bytes, plane stride M*ldr) that the slice-product stage
 * writes.  Bytes not below their modulus give unspecified results.
 */
int alp_emul_crt_bits(int64_t K, int nmoduli);   /* k above; 0 if invalid */

/* The automatic modulus count for C = op(A) op(B) (not in the paper; a
 * heuristic of this library).  Scans the exponents e_i, f_j and, per row of
 * op(A) and column of op(B) with x = |entry| 2^-e, S1 = sum x and S2 = sum x^2;
 * reads back the maxima over rows of 1/S1^2, S2/S1^2, 1/S2 (stats[0..2]) and
 * over columns (stats[3..5]) (one stream synchronisation) and returns in
 * *nmoduli the rule's count (alp_emul_crt_moduli_rule).  workspace: as for
 * alp_gemm_f64_emul with nslices = 0; its sections are overwritten.
 * predicted[0..1] (may be NULL): the rule's predictions for that count. */
alp_status alp_emul_crt_choose(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                               const double* A, int64_t lda, const double* B, int64_t ldb,
                               void* workspace, size_t workspace_bytes, void* stream,
                               int* nmoduli, double* predicted);
/* The rule alone (host only, no GPU): the smallest n in 4..16 with
 * crt_bits(K, n) >= 1 whose predicted largest componentwise error (units of
 * 2^-53, relative to |A||B|; the operand roundings as independent uniform
 * errors, the maximum over M*N elements at sqrt(2 ln(MN)) deviations) is at
 * most half of 0.045 sqrt(K), the native FP64 kernel's modelled error, and
 * whose predicted normwise error is at most half the native kernel's
 * (modelled as 0.311 * 2^-53 * sqrt(S2_i T2_j) per element); else 16.
 * stats[6] as above.  predicted[0] = the componentwise prediction (units of
 * 2^-53), predicted[1] = the normwise ratio to native.  Returns 0 for invalid
 * arguments. */
int alp_emul_crt_moduli_rule(int64_t M, int64_t N, int64_t K, const double* stats,
                             double* predicted);
alp_status alp_emul_recombine_crt(int64_t M, int64_t N, int64_t K, int nmoduli,
                                  const uint8_t* R, int64_t ldr, const int32_t* e,
                                  const int32_t* f, double alpha, double beta, double* C,
                                  int64_t ldc, void* stream);
/* The modular kind's tensor-core stage and reconstruction in one launch
 * (Eq. 1's C = alpha AB + beta C written while the products run): the same C
 * and the same byte planes in R as alp_emul_slice_products followed by
 * alp_emul_recombine_crt, bit for bit.  One persistent launch of CTA pairs
 * takes the 256 x 256 tiles of C from a counter; the product kernel's
 * reconstruction warps rebuild each finished tile from its byte planes while
 * the next tile's products run, and a small second launch rebuilds the tiles
 * of the last wave, whose moduli several pairs share.  alp_gemm_f64_emul runs
 * its modular scheme this way (ALP_EMUL_CRT_FUSE=0 in the environment: as the
 * two stages; the one-block arrangement, ALP_EMUL_CLUSTER=1, always so).
 * da_bf16, db_bf16: the residue slices of A and B^T as alp_emul_split writes
 * them (kpad a multiple of 64, >= K); R: the n byte planes (device, 16-byte
 * aligned, row stride ldr bytes, ldr a multiple of 256 and >= N, plane stride
 * M*ldr), overwritten; e, f: the exponents of the rows of A and the columns
 * of B (device int32); C: row-major M x N (ldc >= N), read when beta != 0;
 * workspace: device memory of alp_emul_products_recombine_crt_workspace(M, N)
 * bytes (4-byte aligned) for the launch's schedule, overwritten.
 * ALP_ERR_INVALID_ARG for K < 1 or an argument the two calls reject,
 * ALP_ERR_WORKSPACE for a missing or short workspace, ALP_ERR_UNSUPPORTED
 * when alp_emul_crt_bits(K, nmoduli) is 0, all before any launch; the device
 * error word reports a wait that gave up. */
size_t alp_emul_products_recombine_crt_workspace(int64_t M, int64_t N);
alp_status alp_emul_products_recombine_crt(int64_t M, int64_t N, int64_t K, int nmoduli,
                                           const void* da_bf16, const void* db_bf16,
                                           int64_t kpad, uint8_t* R, int64_t ldr,
                                           const int32_t* e, const int32_t* f, double alpha,
                                           double beta, double* C, int64_t ldc, void* workspace,
                                           size_t workspace_bytes, void* stream);

/*
 * Emulated FP32 GEMM (the paper evaluates single precision throughout,
 * Sect. 3): C = alpha*A*B + beta*C with float operands, the same digit split,
 * slice products and exact integer sums as alp_gemm_f64_emul, and the result
 * rounded once to float:  X = sum_t S^t 2^(b(nslices+1-t)) (exact, |X| < 2^63),
 * C = (float)alpha * ldexpf(RN_float(X), e_i + f_j - b(nslices+1))
 * (+ fmaf(beta, C, .) when beta != 0).  nslices in 2..4 (nslices * b <= 32);
 * three slices of 8-bit digits (six products) give results within about
 * 0.05 float ulps of |A||B| of the correctly rounded product.  Same
 * workspace layout, kinds, K limits and errors as alp_gemm_f64_emul; floats
 * 4-byte aligned.
 */
alp_status alp_gemm_f32_emul(int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                             int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                             int64_t ldc, int nslices, alp_slice_kind kind, void* workspace,
                             size_t workspace_bytes, void* stream);
size_t alp_gemm_f32_emul_workspace(int64_t M, int64_t N, int64_t K, int nslices,
                                   alp_slice_kind kind);
/* Transposed operands for the emulated GEMMs (BLAS op(X)): C = alpha op(A)
 * op(B) + beta C, op(X) = X for trans 0 and X^T for trans 1.  op(A) is M x K:
 * A is stored M x K (lda >= K) or K x M (lda >= M); op(B) is K x N: B is
 * stored K x N (ldb >= N) or N x K (ldb >= K); all row-major.  Same results
 * bit for bit as alp_gemm_f64_emul / alp_gemm_f32_emul on the transposed
 * matrices; other trans values return ALP_ERR_INVALID_ARG. */
alp_status alp_gemm_f64_emul_ex(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                                double alpha, const double* A, int64_t lda, const double* B,
                                int64_t ldb, double beta, double* C, int64_t ldc, int nslices,
                                alp_slice_kind kind, void* workspace, size_t workspace_bytes,
                                void* stream);
alp_status alp_gemm_f32_emul_ex(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                                float alpha, const float* A, int64_t lda, const float* B,
                                int64_t ldb, float beta, float* C, int64_t ldc, int nslices,
                                alp_slice_kind kind, void* workspace, size_t workspace_bytes,
                                void* stream);
/*
 * Column-major (BLAS) entry points: C = alpha op(A) op(B) + beta C with every
 * matrix column-major: op(A) is M x K with A stored M x K (lda >= M) for
 * trans_a = 0 or K x M (lda >= K) for trans_a = 1; op(B) is K x N with B
 * stored K x N (ldb >= K) or N x K (ldb >= N); C is M x N (ldc >= M).  A
 * column-major matrix is the row-major storage of its transpose, so each call
 * is the row-major call for C^T = op(B)^T op(A)^T: operands, M and N, and the
 * two trans flags swapped (no data is moved for that; the native GEMM packs a
 * row-major-transposed operand as alp_gemm_f64_ex does).  The emulated
 * results equal, bit for bit, those of the row-major calls on the same
 * matrices (each element's scaling exponents and exact product are the same);
 * the native result has the same error bound.  Workspace: the row-major
 * query with swapped arguments, which the *_cm_workspace calls return.
 */
alp_status alp_gemm_f64_cm(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                           double alpha, const double* A, int64_t lda, const double* B,
                           int64_t ldb, double beta, double* C, int64_t ldc,
                           const alp_config* cfg, void* workspace, size_t workspace_bytes,
                           void* stream);
size_t alp_gemm_f64_cm_workspace(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K);
alp_status alp_gemm_f64_emul_cm(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                                double alpha, const double* A, int64_t lda, const double* B,
                                int64_t ldb, double beta, double* C, int64_t ldc, int nslices,
                                alp_slice_kind kind, void* workspace, size_t workspace_bytes,
                                void* stream);
size_t alp_gemm_f64_emul_cm_workspace(int64_t M, int64_t N, int64_t K, int nslices,
                                      alp_slice_kind kind);
alp_status alp_gemm_f32_emul_cm(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                                float alpha, const float* A, int64_t lda, const float* B,
                                int64_t ldb, float beta, float* C, int64_t ldc, int nslices,
                                alp_slice_kind kind, void* workspace, size_t workspace_bytes,
                                void* stream);
size_t alp_gemm_f32_emul_cm_workspace(int64_t M, int64_t N, int64_t K, int nslices,
                                      alp_slice_kind kind);

/* Its stages: the exponent scan and split of alp_emul_exponents and
 * alp_emul_split for float operands (values converted exactly to double), and
 * the FP32 recombination of alp_emul_slice_products' group sums. */
alp_status alp_emul_exponents_f32(int64_t rows, int64_t cols, const float* X, int64_t ldx,
                                  int trans, int32_t* exps, void* stream);
alp_status alp_emul_split_f32(int64_t R, int64_t K, const float* X, int64_t ldx, int trans,
                              const int32_t* exps, int nslices, alp_slice_kind kind,
                              void* out_bf16, int64_t kpad, void* stream);
alp_status alp_emul_recombine_f32(int64_t M, int64_t N, int nslices, alp_slice_kind kind,
                                  const int32_t* G, int64_t ldg, const int32_t* e,
                                  const int32_t* f, float alpha, float beta, float* C,
                                  int64_t ldc, void* stream);

/*
 * Batched variable-size native GEMM: `count` independent problems, each the
 * GEMM of Eq. 1 (Sect. 2, C = alpha A B + beta C) in the row-major form above,
 *   C_p = alpha_p * A_p * B_p + beta_p * C_p,  p = 0..count-1,
 * each problem's C tiles computed as in Sect. 2.1 (one block per C tile,
 * register tiles per thread), with the tile size chosen per size class (the
 * parameter the paper tunes, Sect. 3 / Table 4).
 * All arrays (sizes, scalars, pointers, leading dims) in DEVICE memory, plus
 * HOST copies hM, hN, hK used only to plan tile classes and grid sizes.
 * Every tile of every problem is taken from a device work list by a persistent
 * kernel per size class; the whole call is stream-ordered and capturable in a
 * CUDA graph (see alp_batched_graph_*).  workspace >= alp_gemm_batched_workspace()
 * bytes, 256-byte aligned, owned by the caller.  Errors: negative sizes or a
 * NULL array -> ALP_ERR_INVALID_ARG, a short or misaligned workspace ->
 * ALP_ERR_WORKSPACE, both before any launch.
 */
alp_status alp_gemm_batched_varsize(int64_t count, const int64_t* dM, const int64_t* dN,
                                    const int64_t* dK, const double* dalpha,
                                    const double* const* dA, const int64_t* dlda,
                                    const double* const* dB, const int64_t* dldb,
                                    const double* dbeta, double* const* dC,
                                    const int64_t* dldc, const int64_t* hM,
                                    const int64_t* hN, const int64_t* hK, void* workspace,
                                    size_t workspace_bytes, void* stream);
size_t alp_gemm_batched_workspace(int64_t count, const int64_t* hM, const int64_t* hN,
                                  const int64_t* hK);

/*
 * Autotuner (Sect. 3 "Parameter Tuning": the paper sweeps T per architecture
 * at N = 10240 and keeps the best).  EXHAUSTIVE: times every valid config of
 * `path` on the current GPU (10 CUDA-event-timed runs after warm-up, best
 * kept), appends each timing to the JSONL database (env ALP_TUNE_DB, if set),
 * and caches the winner for (M,N,K,path).  PREDICT: the cost model's argmin
 * over valid configs (ALP_ERR_NOT_TUNED without a loaded model).  LOOKUP:
 * cached winner only.  out: the chosen config; out_tflops: its measured (or
 * for PREDICT, predicted) TFLOP/s, may be NULL.  Allocates its own scratch.
 */
alp_status alp_tune(int64_t M, int64_t N, int64_t K, alp_path path, alp_tune_mode mode,
                    alp_config* out, double* out_tflops);

/* Reads and clears the device error word (synchronises `stream`). */
alp_status alp_get_device_error(void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ALP_H */
