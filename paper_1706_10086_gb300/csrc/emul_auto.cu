// Automatic modulus count of the modular emulated GEMM (nslices = 0 with
// ALP_SLICE_BF16_CRT).  The scheme's only error is the rounding of the scaled
// operands A'_ik = RN(A_ik 2^(k - e_i)) and B'_kj = RN(B_kj 2^(k - f_j)), so
// more moduli (a larger k) make it more accurate and slower.  The count is
// chosen from statistics of the operands' rows and columns, read once by the
// kernels below, with an error model of the scheme and one of the native
// FP64 kernel (both stated at crt_moduli_rule); the choice is a heuristic,
// not a bound.
//
// Statistics, with x = |a| 2^-e for the row's (column's) scale exponent e:
//   S1 = sum |x|, S2 = sum x^2 per row of op(A) and per column of op(B);
//   st[0] = max 1/S1^2, st[1] = max S2/S1^2, st[2] = max 1/S2 over the rows
//   of op(A) (all-zero rows skipped), st[3..5] the same over the columns of
//   op(B).  Accumulated in float (a model input; order does not matter).
#include <cmath>

#include "alp_ext.h"
#include "emul.cuh"

namespace alp {

namespace {

// |a| 2^-e as a float, for |a| < 2^e: exponent and the top 23 mantissa bits
// of the double; 0 for zeros, subnormals, Inf/NaN (the scan reports those) and
// values below float's normal range (negligible in the sums).
__device__ __forceinline__ float scaled_abs_f32(uint64_t bits, int e) {
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0 || ex == 0x7FF) return 0.0f;
    const int fe = ex - 1023 - e + 127;
    if (fe <= 0 || fe >= 255) return 0.0f;
    return __int_as_float((fe << 23) | (int)((bits >> 29) & 0x7FFFFF));
}

// Positive floats order like their bit patterns, so an integer max is a float max.
__device__ __forceinline__ void atomic_max_pos(float* p, float v) {
    atomicMax(reinterpret_cast<int*>(p), __float_as_int(v));
}

__device__ __forceinline__ void record_stats(float s1, float s2, float* out) {
    if (s1 > 0.0f && s2 > 0.0f) {
        atomic_max_pos(out + 0, 1.0f / (s1 * s1));
        atomic_max_pos(out + 1, s2 / (s1 * s1));
        atomic_max_pos(out + 2, 1.0f / s2);
    }
}

// One warp per row of a row-major R x K matrix.
__global__ void crt_stats_rows_kernel(const double* __restrict__ X, int64_t R, int64_t K,
                                      int64_t ldx, const int32_t* __restrict__ e, float* out) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= R) return;
    const double* p = X + row * ldx;
    const int er = e[row];
    float s1 = 0.0f, s2 = 0.0f;
    for (int64_t k = lane; k < K; k += 32) {
        const float x = scaled_abs_f32((uint64_t)__double_as_longlong(__ldg(p + k)), er);
        s1 += x;
        s2 = fmaf(x, x, s2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) record_stats(s1, s2, out);
}

// Columns of a row-major K x N matrix: blocks of 32 columns x 256 rows, 8
// rows in flight per column; partial sums added into s1[N], s2[N].
constexpr int kStatChunk = 256;
__global__ void crt_stats_cols_kernel(const double* __restrict__ X, int64_t K, int64_t N,
                                      int64_t ldx, const int32_t* __restrict__ f,
                                      float* __restrict__ s1, float* __restrict__ s2) {
    __shared__ float r1[8][33], r2[8][33];
    const int64_t j = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.y * kStatChunk;
    const int64_t k1 = (k0 + kStatChunk < K) ? k0 + kStatChunk : K;
    float a1 = 0.0f, a2 = 0.0f;
    if (j < N) {
        const int fj = f[j];
        for (int64_t k = k0 + threadIdx.y; k < k1; k += 8) {
            const float x = scaled_abs_f32((uint64_t)__double_as_longlong(__ldg(X + k * ldx + j)), fj);
            a1 += x;
            a2 = fmaf(x, x, a2);
        }
    }
    r1[threadIdx.y][threadIdx.x] = a1;
    r2[threadIdx.y][threadIdx.x] = a2;
    __syncthreads();
    if (threadIdx.y == 0 && j < N) {
        float t1 = 0.0f, t2 = 0.0f;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            t1 += r1[r][threadIdx.x];
            t2 += r2[r][threadIdx.x];
        }
        atomicAdd(s1 + j, t1);
        atomicAdd(s2 + j, t2);
    }
}

__global__ void crt_stats_finish_kernel(int64_t N, const float* __restrict__ s1,
                                        const float* __restrict__ s2, float* out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) record_stats(s1[j], s2[j], out);
}

// Statistics of the R lines of X (rows of a row-major R x L matrix when
// !trans, else columns of a row-major L x R one), scale exponents `exps`,
// into out[0..2]; s1, s2: R floats of scratch.
alp_status line_stats(const double* X, int64_t R, int64_t L, int64_t ldx, int trans,
                      const int32_t* exps, float* out, float* s1, float* s2, cudaStream_t st) {
    if (R == 0 || L == 0) return ALP_OK;
    if (!trans) {
        const int wpb = 8;
        crt_stats_rows_kernel<<<(unsigned)((R + wpb - 1) / wpb), 32 * wpb, 0, st>>>(X, R, L, ldx,
                                                                                  exps, out);
        return cuda_status(cudaGetLastError());
    }
    if (cudaMemsetAsync(s1, 0, (size_t)R * 4, st) != cudaSuccess ||
        cudaMemsetAsync(s2, 0, (size_t)R * 4, st) != cudaSuccess)
        return ALP_ERR_CUDA;
    const dim3 grid((unsigned)((R + 31) / 32), (unsigned)((L + kStatChunk - 1) / kStatChunk));
    crt_stats_cols_kernel<<<grid, dim3(32, 8), 0, st>>>(X, L, R, ldx, exps, s1, s2);
    crt_stats_finish_kernel<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(R, s1, s2, out);
    return cuda_status(cudaGetLastError());
}

}  // namespace

// The rule.  With u = 2^-53, k = crt_bits(K, n) and the statistics st[6]:
//
//  * the scheme's rounding errors, uniform in half a unit of the scaled
//    operands, give C_ij an error of standard deviation
//    sigma_ij = 2^-k / sqrt(12) * sqrt(4^e_i ||b_j||^2 + 4^f_j ||a_i||^2),
//    and (|A||B|)_ij is about ||a_i||_1 ||b_j||_1 / K, so the largest
//    componentwise error over the M N elements, g = sqrt(2 ln(M N)) standard
//    deviations, is predicted as
//      comp = g / sqrt(12) * 2^(53-k) * K * sqrt(st0 st4 + st3 st1)   [units of u];
//  * the native FP64 kernel's largest componentwise error for operands of
//    one magnitude grows like sqrt(K): modelled as 0.045 sqrt(K) u (4.07 u
//    measured at K = 8192 with this library's DMMA kernel);
//  * normwise, the ratio of the scheme's error to the native kernel's, with
//    the native error modelled as 0.311 u sqrt(K) sqrt(S2_i T2_j / K) per
//    element (calibrated on the same measurement), is
//      norm = 2^(53-k) / (sqrt(12) * 0.311) * sqrt(st2 + st5).
//
// The count is the smallest n with comp <= 0.5 * 0.045 sqrt(K) and norm <=
// 0.5 (half the native kernel's modelled errors, a factor of two against the
// models' own error), else 16.  Operands with an all-zero side give the
// smallest count (the product is exactly zero).
int crt_moduli_rule(int64_t M, int64_t N, int64_t K, const double st[6], double* comp_u,
                    double* norm_ratio) {
    const double kSqrt12 = 3.4641016151377544;
    const double g = std::sqrt(2.0 * std::log((double)(M * N > 2 ? M * N : 2)));
    const double native_comp = 0.045 * std::sqrt((double)(K > 1 ? K : 1));
    const bool zero = !(st[0] > 0.0) || !(st[3] > 0.0);
    int best = 0;
    double c = 0.0, r = 0.0;
    for (int n = kCrtMinModuli; n <= kCrtMaxModuli; ++n) {
        const int k = crt_bits(K, n);
        if (k < 1) continue;
        const double scale = std::ldexp(1.0, 53 - k);
        c = zero ? 0.0 : g / kSqrt12 * scale * (double)K * std::sqrt(st[0] * st[4] + st[3] * st[1]);
        r = zero ? 0.0 : scale / (kSqrt12 * 0.311) * std::sqrt(st[2] + st[5]);
        best = n;
        if (c <= 0.5 * native_comp && r <= 0.5) break;
    }
    if (comp_u) *comp_u = c;
    if (norm_ratio) *norm_ratio = r;
    return best;
}

// Runs the statistics of op(A) and op(B) (exponents e, f already scanned) on
// `stream`, waits for them, and applies the rule.  scratch: 8 + 2 max(M, N)
// floats of device memory.
alp_status crt_choose_moduli(int ta, int tb, int64_t M, int64_t N, int64_t K, const double* A,
                             int64_t lda, const double* B, int64_t ldb, const int32_t* e,
                             const int32_t* f, void* scratch, cudaStream_t stream, int* n_out,
                             double* comp_u, double* norm_ratio) {
    float* out = static_cast<float*>(scratch);
    float* s1 = out + 8;
    float* s2 = s1 + (M > N ? M : N);
    if (cudaMemsetAsync(out, 0, 8 * sizeof(float), stream) != cudaSuccess) return ALP_ERR_CUDA;
    alp_status st;
    // rows of op(A): rows of A, or columns of its K x M storage; columns of
    // op(B): columns of B, or rows of its N x K storage
    if ((st = line_stats(A, M, K, lda, ta, e, out, s1, s2, stream)) != ALP_OK) return st;
    if ((st = line_stats(B, N, K, ldb, 1 - tb, f, out + 3, s1, s2, stream)) != ALP_OK) return st;
    float h[8];
    if (cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return ALP_ERR_CUDA;
    double sd[6];
    for (int i = 0; i < 6; ++i) sd[i] = h[i];
    const int n = crt_moduli_rule(M, N, K, sd, comp_u, norm_ratio);
    if (n < kCrtMinModuli) return ALP_ERR_UNSUPPORTED;
    *n_out = n;
    return ALP_OK;
}

}  // namespace alp

using namespace alp;

extern "C" {

int alp_emul_crt_moduli_rule(int64_t M, int64_t N, int64_t K, const double* stats,
                             double* predicted) {
    if (M < 0 || N < 0 || K < 0 || K > kCrtMaxK || !stats) return 0;
    double c = 0.0, r = 0.0;
    const int n = crt_moduli_rule(M, N, K, stats, &c, &r);
    if (predicted) {
        predicted[0] = c;
        predicted[1] = r;
    }
    return n;
}

}  // extern "C"
