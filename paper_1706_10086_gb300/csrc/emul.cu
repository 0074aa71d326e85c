// Emulated FP64 GEMM (error-free splitting after Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 59, 2012) on BF16 tensor cores:
//
//   1. exponent scan: e_i = frexp exponent of max_k |A_ik|, f_j of max_k |B_kj|
//      (integer max over the IEEE bit patterns; Inf/NaN -> ALP_ERR_UNSUPPORTED);
//   2. split: each A_ik * 2^-e_i is cut into s digits of b = 7 or 8 bits with
//      round half to even (|d_1| <= 2^b, |d_p| <= 2^(b-1)), stored exactly as
//      bf16, K-major for both operands (B is transposed on the way);
//   3. slice products S^t = sum_{p+q=t} D_A^p (D_B^q)^T, t = 2..s+1, on tcgen05
//      (emul_gemm.cu) as exact int32 per group;
//   4. recombination: X = sum_t S^t 2^((s+1-t) b) exactly (128-bit integer),
//      rounded once to the nearest double, scaled by 2^(e_i+f_j-(s+1)b),
//      C = alpha * that (+ fma(beta, C, .)).
//
// Steps 1, 2 and 4 use integer arithmetic on the IEEE encodings and reproduce
// the FP64 definition bit for bit (FP64 arithmetic runs at ~1.1 TFLOP/s on
// this GPU, integer arithmetic far faster).
#include "alp_ext.h"
#include "alp_internal.cuh"
#include "emul.cuh"
#include "emul_split.cuh"

namespace alp {

alp_status native_scale(int64_t M, int64_t N, double beta, double* C, int64_t ldc,
                        cudaStream_t stream);
alp_status validate_gemm(int64_t M, int64_t N, int64_t K, double alpha, const void* A,
                         int64_t lda, const void* B, int64_t ldb, double beta, const void* C,
                         int64_t ldc);
bool select_config(int64_t M, int64_t N, int64_t K, alp_path path, alp_config* out,
                   cudaStream_t stream);
alp_status crt_choose_moduli(int ta, int tb, int64_t M, int64_t N, int64_t K, const double* A,
                             int64_t lda, const double* B, int64_t ldb, const int32_t* e,
                             const int32_t* f, void* scratch, cudaStream_t stream, int* n_out,
                             double* comp_u, double* norm_ratio);

// ---------------------------------------------------------------------------
// 1. exponent scan
// ---------------------------------------------------------------------------
constexpr uint64_t kAbsMask = 0x7FFFFFFFFFFFFFFFull;


// |x| as ordered integer keys (larger key, larger |x|): the bits of a double
// without its sign, or of a float.  A key at or above the infinity's is Inf
// or NaN.  The float key converts to the double bits of the same value for
// the exponent (FP32 operands convert exactly, so frexp and the digits are
// the same as for the double of equal value).
template <typename T> struct ScanKey;
template <> struct ScanKey<double> {
    using type = uint64_t;
    static constexpr uint64_t kInf = 0x7FF0000000000000ull;
    __device__ static uint64_t of(uint64_t bits) { return bits & kAbsMask; }
    __device__ static uint64_t to_double_bits(uint64_t k) { return k; }
};
template <> struct ScanKey<float> {
    using type = uint32_t;
    static constexpr uint32_t kInf = 0x7F800000u;
    __device__ static uint32_t of(uint32_t bits) { return bits & 0x7FFFFFFFu; }
    __device__ static uint64_t to_double_bits(uint32_t k) {
        return (uint64_t)__double_as_longlong((double)__int_as_float((int)k));
    }
};

// Largest key of the V = 16 / sizeof(T) elements of a 16-byte vector.
template <typename T>
__device__ __forceinline__ typename ScanKey<T>::type vec_key(uint4 v) {
    using SK = ScanKey<T>;
    if constexpr (sizeof(T) == 8) {
        const uint64_t a = SK::of(((uint64_t)v.y << 32) | v.x);
        const uint64_t b = SK::of(((uint64_t)v.w << 32) | v.z);
        return a > b ? a : b;
    } else {
        const uint32_t a = max(SK::of(v.x), SK::of(v.y)), b = max(SK::of(v.z), SK::of(v.w));
        return max(a, b);
    }
}
template <typename T>
__device__ __forceinline__ typename ScanKey<T>::type elem_key(const T* p) {
    using SK = ScanKey<T>;
    if constexpr (sizeof(T) == 8) return SK::of((uint64_t)__double_as_longlong(__ldg(p)));
    else return SK::of((uint32_t)__float_as_int(__ldg(p)));
}

// One warp per row of a row-major R x K matrix (T = double or float): the
// 16-byte aligned body as vectors, four in flight per lane; the ragged ends
// element by element.
template <typename T>
__global__ void scan_rows_kernel(const T* __restrict__ X, int64_t R, int64_t K, int64_t ldx,
                                 int32_t* __restrict__ e, int* err) {
    using SK = ScanKey<T>;
    using Key = typename SK::type;
    constexpr int V = 16 / (int)sizeof(T);
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= R) return;
    const T* p = X + row * ldx;
    int64_t head = (int64_t)(((16 - (reinterpret_cast<uintptr_t>(p) & 15)) & 15) / sizeof(T));
    if (head > K) head = K;
    const int64_t nvec = (K - head) / V;
    Key mx = 0;
    if (lane < head) mx = elem_key(p + lane);
    const uint4* pv = reinterpret_cast<const uint4*>(p + head);
    int64_t v = lane;
    for (; v + 96 < nvec; v += 128) {
        const uint4 a = __ldg(pv + v), b = __ldg(pv + v + 32), c = __ldg(pv + v + 64),
                    d = __ldg(pv + v + 96);
        const Key ka = vec_key<T>(a), kb = vec_key<T>(b), kc = vec_key<T>(c), kd = vec_key<T>(d);
        const Key k1 = ka > kb ? ka : kb, k2 = kc > kd ? kc : kd;
        const Key k3 = k1 > k2 ? k1 : k2;
        mx = k3 > mx ? k3 : mx;
    }
    for (; v < nvec; v += 32) {
        const Key k1 = vec_key<T>(__ldg(pv + v));
        mx = k1 > mx ? k1 : mx;
    }
    for (int64_t k = head + nvec * V + lane; k < K; k += 32) {
        const Key k1 = elem_key(p + k);
        mx = k1 > mx ? k1 : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const Key y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    if (lane == 0) {
        if (mx >= SK::kInf) set_device_error(err, ALP_ERR_UNSUPPORTED);
        e[row] = frexp_exponent_of_bits(SK::to_double_bits(mx));
    }
}

// Columns of a row-major K x N matrix: blocks of 32 x V columns (one 16-byte
// vector per thread; element by element where a vector would leave the row
// or is unaligned) x (8 threads x kColChunk rows), four rows in flight per
// thread.  The frexp exponent grows with |x|, so the column exponent is the
// atomic max of the blocks' exponents; f starts at kNoExp (memset to 0x80
// bytes) and all-zero columns are set to 0 afterwards.
constexpr int kColChunk = 256;
constexpr int32_t kNoExp = (int32_t)0x80808080;

template <typename T>
__global__ void scan_cols_kernel(const T* __restrict__ X, int64_t K, int64_t N, int64_t ldx,
                                 int32_t* __restrict__ f, int* err) {
    using SK = ScanKey<T>;
    using Key = typename SK::type;
    constexpr int V = 16 / (int)sizeof(T);
    __shared__ Key red[8][32 * V];
    const int64_t j = ((int64_t)blockIdx.x * 32 + threadIdx.x) * V;
    const int64_t k0 = (int64_t)blockIdx.y * kColChunk;
    const int64_t k1 = (k0 + kColChunk < K) ? k0 + kColChunk : K;
    Key mx[V];
#pragma unroll
    for (int c = 0; c < V; ++c) mx[c] = 0;
    const bool vec = j + V <= N && (reinterpret_cast<uintptr_t>(X + j) & 15) == 0 &&
                     ((ldx * (int64_t)sizeof(T)) & 15) == 0;
    if (vec) {
        int64_t k = k0 + threadIdx.y;
        for (; k + 24 < k1; k += 32) {
            uint4 w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                w[q] = __ldg(reinterpret_cast<const uint4*>(X + (k + 8 * q) * ldx + j));
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t* u = reinterpret_cast<const uint32_t*>(&w[q]);
#pragma unroll
                for (int c = 0; c < V; ++c) {
                    Key kk;
                    if constexpr (sizeof(T) == 8)
                        kk = SK::of(((uint64_t)u[2 * c + 1] << 32) | u[2 * c]);
                    else
                        kk = SK::of(u[c]);
                    mx[c] = kk > mx[c] ? kk : mx[c];
                }
            }
        }
        for (; k < k1; k += 8) {
            const uint4 w = __ldg(reinterpret_cast<const uint4*>(X + k * ldx + j));
            const uint32_t* u = reinterpret_cast<const uint32_t*>(&w);
#pragma unroll
            for (int c = 0; c < V; ++c) {
                Key kk;
                if constexpr (sizeof(T) == 8) kk = SK::of(((uint64_t)u[2 * c + 1] << 32) | u[2 * c]);
                else kk = SK::of(u[c]);
                mx[c] = kk > mx[c] ? kk : mx[c];
            }
        }
    } else {
        for (int64_t k = k0 + threadIdx.y; k < k1; k += 8)
#pragma unroll
            for (int c = 0; c < V; ++c)
                if (j + c < N) {
                    const Key kk = elem_key(X + k * ldx + j + c);
                    mx[c] = kk > mx[c] ? kk : mx[c];
                }
    }
    bool bad = false;
#pragma unroll
    for (int c = 0; c < V; ++c) {
        red[threadIdx.y][threadIdx.x * V + c] = mx[c];
        bad |= mx[c] >= SK::kInf;
    }
    if (bad) set_device_error(err, ALP_ERR_UNSUPPORTED);
    __syncthreads();
    // the block's 32 V columns, 8 partial maxima each: thread tid finishes
    // column tid (threads beyond 32 V have none)
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int col = tid; col < 32 * V; col += 256) {
        const int64_t jc = (int64_t)blockIdx.x * 32 * V + col;
        if (jc >= N) continue;
        Key m = red[0][col];
#pragma unroll
        for (int r = 1; r < 8; ++r) m = red[r][col] > m ? red[r][col] : m;
        if (m && m < SK::kInf) atomicMax(f + jc, frexp_exponent_of_bits(SK::to_double_bits(m)));
    }
}

__global__ void zero_empty_columns_kernel(int64_t N, int32_t* __restrict__ f) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N && f[j] == kNoExp) f[j] = 0;
}

// ---------------------------------------------------------------------------
// 4. recombination + alpha/beta epilogue
// ---------------------------------------------------------------------------
// X = sum_t v[t] 2^(B (S-1-t)) exactly (Horner, X = X * 2^B + v[t]), then the
// nearest double times 2^E.  The first terms run in 64 bits (after t + 1 terms
// |X| < 2^(32 + B t)); the rest carry a 128-bit hi:lo pair.
template <int S, int B>
__device__ __forceinline__ double recombine_vals(const int32_t (&v)[S], int E) {
    constexpr int T64 = (62 - 32) / B + 1;   // terms that fit in 64 bits
    int64_t x = v[0];
#pragma unroll
    for (int t = 1; t < (S < T64 ? S : T64); ++t) x = x * (1ll << B) + v[t];
    int64_t hi = x >> 63;
    uint64_t lo = (uint64_t)x;
#pragma unroll
    for (int t = T64; t < S; ++t) {
        const uint64_t l2 = lo << B;
        const uint64_t h2 = ((uint64_t)hi << B) | (lo >> (64 - B));
        const int64_t vt = v[t];
        uint64_t rlo, rhi;
        asm("add.cc.u64 %0, %2, %4;\n\taddc.u64 %1, %3, %5;"
            : "=l"(rlo), "=l"(rhi)
            : "l"(l2), "l"(h2), "l"((uint64_t)vt), "l"((uint64_t)(vt >> 63)));
        lo = rlo;
        hi = (int64_t)rhi;
    }
    return i128_scaled_to_double_rn(hi, lo, E);
}

// One block row of threads per matrix row chunk: rows from blockIdx.y (grid
// stride), two columns per thread from the x dimension (no integer division
// per element).
template <int S, int B>
__device__ __forceinline__ double recombine_one(const int32_t* __restrict__ g, int64_t gplane,
                                                int E) {
    int32_t v[S];
#pragma unroll
    for (int t = 0; t < S; ++t) v[t] = __ldg(g + (int64_t)t * gplane);
    return recombine_vals<S, B>(v, E);
}

template <int S, int B>
__global__ void recombine_kernel(const int32_t* __restrict__ G, int64_t gplane, int64_t ldg,
                                 const int32_t* __restrict__ e, const int32_t* __restrict__ f,
                                 int64_t M, int64_t N, double alpha, double beta,
                                 double* __restrict__ C, int64_t ldc) {
    const int shift0 = (S + 1) * B;
    for (int64_t i = blockIdx.y; i < M; i += gridDim.y) {
        const int ei = e[i] - shift0;
        const int32_t* gi = G + i * ldg;
        double* ci = C + i * ldc;
        for (int64_t j = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); j < N;
             j += 2 * (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int64_t jj = j + u;
                if (jj >= N) break;
                const double w = recombine_one<S, B>(gi + jj, gplane, ei + __ldg(f + jj));
                double out = (alpha == 1.0) ? w : (alpha == -1.0) ? -w : alpha * w;
                if (beta != 0.0) out = __fma_rn(beta, ci[jj], out);
                ci[jj] = out;
            }
        }
    }
}

// Four columns per thread: the S group sums of four adjacent columns arrive
// as one 16-byte load per plane (G rows are 256-column padded, so the vector
// never leaves the row), and C is written as two 16-byte stores when the row
// of C is 16-byte aligned.  Needs G 16-byte aligned (the launch checks).
template <int S, int B>
__global__ void __launch_bounds__(256) recombine4_kernel(
    const int32_t* __restrict__ G, int64_t gplane, int64_t ldg, const int32_t* __restrict__ e,
    const int32_t* __restrict__ f, int64_t M, int64_t N, double alpha, double beta,
    double* __restrict__ C, int64_t ldc) {
    const int shift0 = (S + 1) * B;
    for (int64_t i = blockIdx.y; i < M; i += gridDim.y) {
        const int ei = e[i] - shift0;
        const int32_t* gi = G + i * ldg;
        double* ci = C + i * ldc;
        const bool cvec = (reinterpret_cast<uintptr_t>(ci) & 15) == 0;
        for (int64_t j = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); j < N;
             j += 4 * (int64_t)gridDim.x * blockDim.x) {
            int4 v[S];
#pragma unroll
            for (int t = 0; t < S; ++t)
                v[t] = __ldg(reinterpret_cast<const int4*>(gi + (int64_t)t * gplane + j));
            double out[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (j + u >= N) break;
                int32_t c[S];
#pragma unroll
                for (int t = 0; t < S; ++t)
                    c[t] = u == 0 ? v[t].x : u == 1 ? v[t].y : u == 2 ? v[t].z : v[t].w;
                const double w = recombine_vals<S, B>(c, ei + __ldg(f + j + u));
                double o = (alpha == 1.0) ? w : (alpha == -1.0) ? -w : alpha * w;
                if (beta != 0.0) o = __fma_rn(beta, ci[j + u], o);
                out[u] = o;
            }
            if (cvec && j + 3 < N) {
                reinterpret_cast<double2*>(ci + j)[0] = make_double2(out[0], out[1]);
                reinterpret_cast<double2*>(ci + j)[1] = make_double2(out[2], out[3]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (j + u < N) ci[j + u] = out[u];
            }
        }
    }
}

template <int B>
static alp_status launch_recombine_b(int s, dim3 grid, cudaStream_t st, const int32_t* G,
                                     int64_t gplane, int64_t ldg, const int32_t* e,
                                     const int32_t* f, int64_t M, int64_t N, double alpha,
                                     double beta, double* C, int64_t ldc) {
    const bool vec = (reinterpret_cast<uintptr_t>(G) & 15) == 0 && gplane % 4 == 0 && ldg % 4 == 0;
    if (vec) grid.x = (unsigned)((grid.x + 1) / 2);   // four columns per thread instead of two
#define ALP_RECOMBINE_CASE(x)                                                                     \
    case x:                                                                                      \
        if (vec)                                                                                 \
            recombine4_kernel<x, B><<<grid, 256, 0, st>>>(G, gplane, ldg, e, f, M, N, alpha, beta, \
                                                          C, ldc);                               \
        else                                                                                     \
            recombine_kernel<x, B><<<grid, 256, 0, st>>>(G, gplane, ldg, e, f, M, N, alpha, beta,  \
                                                         C, ldc);                                \
        break;
    switch (s) {
        ALP_RECOMBINE_CASE(1) ALP_RECOMBINE_CASE(2) ALP_RECOMBINE_CASE(3) ALP_RECOMBINE_CASE(4)
        ALP_RECOMBINE_CASE(5) ALP_RECOMBINE_CASE(6) ALP_RECOMBINE_CASE(7) ALP_RECOMBINE_CASE(8)
        default: return ALP_ERR_INVALID_ARG;
    }
#undef ALP_RECOMBINE_CASE
    return cuda_status(cudaGetLastError());
}

static alp_status launch_recombine(int s, int b, dim3 grid, cudaStream_t st, const int32_t* G,
                                   int64_t gplane, int64_t ldg, const int32_t* e, const int32_t* f,
                                   int64_t M, int64_t N, double alpha, double beta, double* C,
                                   int64_t ldc) {
    if (b == 7)
        return launch_recombine_b<7>(s, grid, st, G, gplane, ldg, e, f, M, N, alpha, beta, C, ldc);
    if (b == 8)
        return launch_recombine_b<8>(s, grid, st, G, gplane, ldg, e, f, M, N, alpha, beta, C, ldc);
    return ALP_ERR_INVALID_ARG;
}

dim3 recombine_grid(int64_t M, int64_t N) {
    const int64_t bx = (N + 511) / 512;
    int64_t by = (int64_t)device_sm_count() * 16 / (bx > 0 ? bx : 1);
    if (by < 1) by = 1;
    if (by > M) by = M;
    if (by > 65535) by = 65535;
    return dim3((unsigned)(bx > 0 ? bx : 1), (unsigned)by);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

EmulLayout emul_layout(int64_t M, int64_t N, int64_t K, int s, int gbytes) {
    EmulLayout L;
    L.kpad = (K + kEmulBK - 1) / kEmulBK * kEmulBK;
    if (L.kpad == 0) L.kpad = kEmulBK;
    L.ldg = (N + 255) / 256 * 256;   // whole 256-column tiles per row (emul_gemm stores)
    size_t off = 0;
    L.off_da = off; off += up256((size_t)s * M * L.kpad * 2);
    L.off_db = off; off += up256((size_t)s * N * L.kpad * 2);
    L.off_g = off;  off += up256((size_t)s * M * L.ldg * gbytes);
    L.off_e = off; off += up256((size_t)M * 4);
    L.off_f = off; off += up256((size_t)N * 4);
    L.off_sched = off;
    L.sched_bytes = gbytes == 1 ? emul_crt_sched_bytes(M, N) : 0;
    off += up256(L.sched_bytes);
    L.bytes = off;
    return L;
}

static int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
alp_status emul_exponents(int64_t rows, int64_t cols, const T* X, int64_t ldx, int trans,
                          int32_t* exps, cudaStream_t st) {
    int* err = device_error_word();
    if (!trans) {
        const int wpb = 8;
        scan_rows_kernel<T><<<(unsigned)((rows + wpb - 1) / wpb), 32 * wpb, 0, st>>>(
            X, rows, cols, ldx, exps, err);
        return cuda_status(cudaGetLastError());
    }
    // trans: X is cols x rows row-major (K x N); exponents per column (rows = N)
    const int64_t N = rows, K = cols;
    if (cudaMemsetAsync(exps, 0x80, (size_t)N * 4, st) != cudaSuccess) return ALP_ERR_CUDA;
    constexpr int V = 16 / (int)sizeof(T);
    dim3 grid((unsigned)((N + 32 * V - 1) / (32 * V)), (unsigned)((K + kColChunk - 1) / kColChunk));
    if (K > 0) scan_cols_kernel<T><<<grid, dim3(32, 8), 0, st>>>(X, K, N, ldx, exps, err);
    zero_empty_columns_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, exps);
    return cuda_status(cudaGetLastError());
}

template <typename T, int B>
static alp_status emul_split_b(int64_t R, int64_t K, const T* X, int64_t ldx, int trans,
                               const int32_t* exps, int s, __nv_bfloat16* out, int64_t kpad,
                               cudaStream_t st) {
    const bool vec = (reinterpret_cast<uintptr_t>(out) & 7) == 0 && kpad % 4 == 0;
    const int64_t bx = (kpad + 1023) / 1024;
    int64_t by = (int64_t)device_sm_count() * 8 / bx;
    by = by < 1 ? 1 : by > R ? R : by > 65535 ? 65535 : by;
    const dim3 grid4((unsigned)bx, (unsigned)by);
#define ALP_SPLIT_CASE(x)                                                                        \
    case x:                                                                                      \
        if (!trans && vec)                                                                       \
            split_rows4_kernel<T, x, DigitSplit<B>><<<grid4, 256, 0, st>>>(X, R, K, ldx, exps,  \
                                                                           out, kpad, {});    \
        else if (!trans)                                                                         \
            split_rows_kernel<T, x, DigitSplit<B>><<<grid_for(R * (kpad / 2), 256), 256, 0, st>>>( \
                X, R, K, ldx, exps, out, kpad, {});                                              \
        else                                                                                     \
            split_cols_kernel<T, x, DigitSplit<B>><<<dim3((unsigned)((R + 31) / 32),              \
                                                          (unsigned)(kpad / 64)),                \
                                      256, 0, st>>>(X, K, R, ldx, exps, out, kpad, {});          \
        break;
    switch (s) {
        ALP_SPLIT_CASE(1) ALP_SPLIT_CASE(2) ALP_SPLIT_CASE(3) ALP_SPLIT_CASE(4)
        ALP_SPLIT_CASE(5) ALP_SPLIT_CASE(6) ALP_SPLIT_CASE(7) ALP_SPLIT_CASE(8)
        default: return ALP_ERR_INVALID_ARG;
    }
#undef ALP_SPLIT_CASE
    return cuda_status(cudaGetLastError());
}

template <typename T>
alp_status emul_split(int64_t R, int64_t K, const T* X, int64_t ldx, int trans,
                      const int32_t* exps, int s, __nv_bfloat16* out, int64_t kpad,
                      cudaStream_t st, int b) {
    if (b == 7) return emul_split_b<T, 7>(R, K, X, ldx, trans, exps, s, out, kpad, st);
    if (b == 8) return emul_split_b<T, 8>(R, K, X, ldx, trans, exps, s, out, kpad, st);
    return ALP_ERR_INVALID_ARG;
}

// ---------------------------------------------------------------------------
// FP32 results (alp_gemm_f32_emul): with s b <= 32 the exact sum X fits in 64
// bits; it is rounded once to float (cvt.rn.f32.s64), scaled by 2^E (by the
// exponent field while the result stays normal, else by ldexpf, which rounds
// a subnormal result a second time, as the definition does), then alpha and
// the fused beta term in float.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float i64_scaled_to_float_rn(int64_t x, int E) {
    float v;
    asm("cvt.rn.f32.s64 %0, %1;" : "=f"(v) : "l"(x));
    if (v == 0.0f) return v;
    const uint32_t bits = __float_as_uint(v);
    const int ne = (int)((bits >> 23) & 0xFF) + E;
    if (ne >= 1 && ne <= 254) return __uint_as_float((bits & 0x807FFFFFu) | ((uint32_t)ne << 23));
    return ldexpf(v, E);
}

template <int S, int B>
__global__ void __launch_bounds__(256) recombine_f32_kernel(
    const int32_t* __restrict__ G, int64_t gplane, int64_t ldg, const int32_t* __restrict__ e,
    const int32_t* __restrict__ f, int64_t M, int64_t N, float alpha, float beta,
    float* __restrict__ C, int64_t ldc, bool gvec) {
    const int shift0 = (S + 1) * B;
    for (int64_t i = blockIdx.y; i < M; i += gridDim.y) {
        const int ei = e[i] - shift0;
        const int32_t* gi = G + i * ldg;
        float* ci = C + i * ldc;
        const bool cvec = (reinterpret_cast<uintptr_t>(ci) & 15) == 0;
        for (int64_t j = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); j < N;
             j += 4 * (int64_t)gridDim.x * blockDim.x) {
            int4 v[S];
#pragma unroll
            for (int t = 0; t < S; ++t) {
                const int32_t* g = gi + (int64_t)t * gplane + j;
                if (gvec) {   // ldg and j are multiples of 4: the vector stays in the row
                    v[t] = __ldg(reinterpret_cast<const int4*>(g));
                } else {      // element by element, nothing read past column N - 1
                    v[t] = make_int4(__ldg(g), j + 1 < N ? __ldg(g + 1) : 0,
                                     j + 2 < N ? __ldg(g + 2) : 0, j + 3 < N ? __ldg(g + 3) : 0);
                }
            }
            float out[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (j + u >= N) break;
                int64_t X = 0;
#pragma unroll
                for (int t = 0; t < S; ++t) {
                    const int32_t c = u == 0 ? v[t].x : u == 1 ? v[t].y : u == 2 ? v[t].z : v[t].w;
                    X = X * (1ll << B) + c;
                }
                const float w = i64_scaled_to_float_rn(X, ei + __ldg(f + j + u));
                float o = (alpha == 1.0f) ? w : (alpha == -1.0f) ? -w : __fmul_rn(alpha, w);
                if (beta != 0.0f) o = __fmaf_rn(beta, ci[j + u], o);
                out[u] = o;
            }
            if (cvec && j + 3 < N) {
                *reinterpret_cast<float4*>(ci + j) = make_float4(out[0], out[1], out[2], out[3]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (j + u < N) ci[j + u] = out[u];
            }
        }
    }
}

template <int B>
static alp_status launch_recombine_f32_b(int s, dim3 grid, cudaStream_t st, const int32_t* G,
                                         int64_t gplane, int64_t ldg, const int32_t* e,
                                         const int32_t* f, int64_t M, int64_t N, float alpha,
                                         float beta, float* C, int64_t ldc) {
    const bool gvec = (reinterpret_cast<uintptr_t>(G) & 15) == 0 && gplane % 4 == 0 && ldg % 4 == 0;
    grid.x = (unsigned)((grid.x + 1) / 2);   // four columns per thread
#define ALP_RECOMBINE_F32_CASE(x)                                                                 \
    case x:                                                                                      \
        recombine_f32_kernel<x, B><<<grid, 256, 0, st>>>(G, gplane, ldg, e, f, M, N, alpha, beta,  \
                                                         C, ldc, gvec);                          \
        break;
    switch (s) {
        ALP_RECOMBINE_F32_CASE(1) ALP_RECOMBINE_F32_CASE(2) ALP_RECOMBINE_F32_CASE(3)
        ALP_RECOMBINE_F32_CASE(4)
        default: return ALP_ERR_INVALID_ARG;
    }
#undef ALP_RECOMBINE_F32_CASE
    return cuda_status(cudaGetLastError());
}

static alp_status launch_recombine_f32(int s, int b, dim3 grid, cudaStream_t st, const int32_t* G,
                                       int64_t gplane, int64_t ldg, const int32_t* e,
                                       const int32_t* f, int64_t M, int64_t N, float alpha,
                                       float beta, float* C, int64_t ldc) {
    if (b == 7)
        return launch_recombine_f32_b<7>(s, grid, st, G, gplane, ldg, e, f, M, N, alpha, beta, C, ldc);
    if (b == 8)
        return launch_recombine_f32_b<8>(s, grid, st, G, gplane, ldg, e, f, M, N, alpha, beta, C, ldc);
    return ALP_ERR_INVALID_ARG;
}

// C = beta C for FP32 (alpha == 0 or K == 0): beta == 0 writes zeros.
__global__ void scale_f32_kernel(float* __restrict__ C, int64_t ldc, int64_t M, int64_t N,
                                 float beta) {
    const int64_t total = M * N;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / N, j = idx - i * N;
        float* c = C + i * ldc + j;
        *c = beta == 0.0f ? 0.0f : __fmul_rn(beta, *c);
    }
}

// The emulated GEMM for double or float operands: C = alpha op(A) op(B) +
// beta C with op(X) = X (trans 0) or X^T (trans 1).  A transposed A is split
// by columns of its storage and a transposed B by rows, which is the K-major
// digit layout the tensor-core stage reads, so transposes cost nothing.
template <typename T>
alp_status emul_gemm_impl(int ta, int tb, int64_t M, int64_t N, int64_t K, T alpha, const T* A,
                          int64_t lda, const T* B, int64_t ldb, T beta, T* C, int64_t ldc,
                          int nslices, alp_slice_kind kind, void* workspace,
                          size_t workspace_bytes, cudaStream_t s) {
    constexpr bool kF32 = sizeof(T) == 4;
    if (M < 0 || N < 0 || K < 0 || (ta != 0 && ta != 1) || (tb != 0 && tb != 1))
        return ALP_ERR_INVALID_ARG;
    if (kind == ALP_SLICE_INT8) return ALP_ERR_UNSUPPORTED;   // no tcgen05 kind::i8 on sm_103a
    EmulScheme sc;
    if (!emul_scheme_of(kind, &sc)) return ALP_ERR_INVALID_ARG;
    if (kF32 && sc.crt) return ALP_ERR_UNSUPPORTED;           // the modular scheme is FP64 only
    const int b = sc.b;
    // nslices = 0 with the modular scheme: the count is chosen from the
    // operands (emul_auto.cu) once their exponents are known
    const bool auto_n = !kF32 && sc.crt && nslices == 0;
    if (!auto_n && !emul_slices_ok(sc, nslices, kF32)) return ALP_ERR_INVALID_ARG;
    if (M == 0 || N == 0) return ALP_OK;
    if (lda < (ta ? M : K) || ldb < (tb ? K : N) || ldc < N || !C) return ALP_ERR_INVALID_ARG;
    const bool reads_ab = alpha != T(0) && K > 0;
    if (reads_ab && (!A || !B)) return ALP_ERR_INVALID_ARG;
    if (((uintptr_t)C % sizeof(T)) ||
        (reads_ab && (((uintptr_t)A % sizeof(T)) || ((uintptr_t)B % sizeof(T)))))
        return ALP_ERR_INVALID_ARG;   // elements must be naturally aligned
    if (!reads_ab) {
        if constexpr (kF32) {
            int64_t blocks = (M * N + 255) / 256;
            const int64_t cap = (int64_t)device_sm_count() * 8;
            blocks = blocks > cap ? cap : blocks < 1 ? 1 : blocks;
            scale_f32_kernel<<<(unsigned)blocks, 256, 0, s>>>(C, ldc, M, N, beta);
            return cuda_status(cudaGetLastError());
        } else {
            return native_scale(M, N, beta, C, ldc, s);
        }
    }
    if (K > emul_scheme_max_k(sc) || M > 0x7fffffffLL || N > 0x7fffffffLL)
        return ALP_ERR_UNSUPPORTED;
    // with an automatic count the workspace is laid out for the most moduli;
    // e and f stay where that layout puts them, beyond every section of the
    // chosen count's layout
    const EmulLayout L0 = emul_layout(M, N, K, auto_n ? kCrtMaxModuli : nslices, sc.crt ? 1 : 4);
    if (!workspace || workspace_bytes < L0.bytes || ((uintptr_t)workspace & 255))
        return ALP_ERR_WORKSPACE;
    if (!auto_n && sc.crt && crt_bits(K, nslices) < 1) return ALP_ERR_UNSUPPORTED;
    char* ws = static_cast<char*>(workspace);
    auto* e = reinterpret_cast<int32_t*>(ws + L0.off_e);
    auto* f = reinterpret_cast<int32_t*>(ws + L0.off_f);
    // rows of op(A): rows of A, or columns of its K x M storage; columns of
    // op(B): columns of B, or rows of its N x K storage
    alp_status st;
    // the modular scheme with a given count and A not transposed scans A's
    // rows inside its split (emul_scan_split_crt), after B's scan
    bool fused_a = false;
    if constexpr (!kF32) fused_a = sc.crt && !auto_n && ta == 0;
    if (!fused_a && (st = emul_exponents(M, K, A, lda, ta, e, s)) != ALP_OK) return st;
    if ((st = emul_exponents(N, K, B, ldb, 1 - tb, f, s)) != ALP_OK) return st;
    if constexpr (!kF32) {
        if (auto_n) {   // statistics in the (not yet written) residue-byte section
            if ((st = crt_choose_moduli(ta, tb, M, N, K, A, lda, B, ldb, e, f, ws + L0.off_g, s,
                                        &nslices, nullptr, nullptr)) != ALP_OK)
                return st;
        }
    }
    const int kcrt = sc.crt ? crt_bits(K, nslices) : 0;
    if (sc.crt && kcrt < 1) return ALP_ERR_UNSUPPORTED;
    const EmulLayout L = auto_n ? emul_layout(M, N, K, nslices, 1) : L0;
    auto* da = reinterpret_cast<__nv_bfloat16*>(ws + L.off_da);
    auto* db = reinterpret_cast<__nv_bfloat16*>(ws + L.off_db);
    auto* G = reinterpret_cast<int32_t*>(ws + L.off_g);
    if constexpr (kF32) {
        if ((st = emul_split(M, K, A, lda, ta, e, nslices, da, L.kpad, s, b)) != ALP_OK) return st;
        if ((st = emul_split(N, K, B, ldb, 1 - tb, f, nslices, db, L.kpad, s, b)) != ALP_OK)
            return st;
    } else if (sc.crt) {
        if ((st = fused_a ? emul_scan_split_crt(M, K, A, lda, e, nslices, da, L.kpad, kcrt, s)
                          : emul_split_crt(M, K, A, lda, ta, e, nslices, da, L.kpad, kcrt, s)) !=
            ALP_OK)
            return st;
        if ((st = emul_split_crt(N, K, B, ldb, 1 - tb, f, nslices, db, L.kpad, kcrt, s)) != ALP_OK)
            return st;
    } else {
        if ((st = emul_split(M, K, A, lda, ta, e, nslices, da, L.kpad, s, b)) != ALP_OK) return st;
        if ((st = emul_split(N, K, B, ldb, 1 - tb, f, nslices, db, L.kpad, s, b)) != ALP_OK)
            return st;
    }
    alp_config cfg;
    const bool have = select_config(M, N, K, ALP_PATH_EMUL, &cfg, s) && emul_config_valid(cfg);
    if constexpr (!kF32) {
        if (sc.crt)   // products and reconstruction (one launch with CTA pairs)
            return emul_crt_products_recombine(
                M, N, K, nslices, da, db, L.kpad, reinterpret_cast<uint8_t*>(G), L.ldg, e, f,
                kcrt, alpha, beta, C, ldc, reinterpret_cast<int*>(ws + L0.off_sched),
                L0.sched_bytes, s, have ? cfg.stages : 0, have ? emul_arrangement_of(cfg) : 0);
    }
    if ((st = emul_slice_gemm(M, N, K, nslices, da, db, L.kpad, G, L.ldg, s,
                              have ? cfg.stages : 0, have ? emul_arrangement_of(cfg) : 0, b,
                              sc.trim, sc.crt)) != ALP_OK)
        return st;
    if constexpr (kF32)
        return launch_recombine_f32(nslices, b, recombine_grid(M, N), s, G, M * L.ldg, L.ldg, e,
                                    f, M, N, alpha, beta, C, ldc);
    else
        return launch_recombine(nslices, b, recombine_grid(M, N), s, G, M * L.ldg, L.ldg, e, f,
                                M, N, alpha, beta, C, ldc);
}

}  // namespace alp

using namespace alp;

extern "C" {

size_t alp_gemm_f64_emul_workspace(int64_t M, int64_t N, int64_t K, int nslices,
                                   alp_slice_kind kind) {
    EmulScheme sc;
    if (M < 0 || N < 0 || K < 0 || !emul_scheme_of(kind, &sc)) return 0;
    if (sc.crt && nslices == 0) return emul_layout(M, N, K, kCrtMaxModuli, 1).bytes;
    if (!emul_slices_ok(sc, nslices, false)) return 0;
    return emul_layout(M, N, K, nslices, sc.crt ? 1 : 4).bytes;
}

alp_status alp_emul_crt_choose(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                               const double* A, int64_t lda, const double* B, int64_t ldb,
                               void* workspace, size_t workspace_bytes, void* stream,
                               int* nmoduli, double* predicted) {
    if (M < 0 || N < 0 || K < 0 || (trans_a != 0 && trans_a != 1) ||
        (trans_b != 0 && trans_b != 1) || !nmoduli)
        return ALP_ERR_INVALID_ARG;
    if (K > kCrtMaxK || M > 0x7fffffffLL || N > 0x7fffffffLL) return ALP_ERR_UNSUPPORTED;
    if (M == 0 || N == 0 || K == 0) {
        *nmoduli = kCrtMinModuli;
        if (predicted) predicted[0] = predicted[1] = 0.0;
        return ALP_OK;
    }
    if (!A || !B || lda < (trans_a ? M : K) || ldb < (trans_b ? K : N)) return ALP_ERR_INVALID_ARG;
    const EmulLayout L0 = emul_layout(M, N, K, kCrtMaxModuli, 1);
    if (!workspace || workspace_bytes < L0.bytes || ((uintptr_t)workspace & 255))
        return ALP_ERR_WORKSPACE;
    char* ws = static_cast<char*>(workspace);
    auto* e = reinterpret_cast<int32_t*>(ws + L0.off_e);
    auto* f = reinterpret_cast<int32_t*>(ws + L0.off_f);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    alp_status st;
    if ((st = emul_exponents(M, K, A, lda, trans_a, e, s)) != ALP_OK) return st;
    if ((st = emul_exponents(N, K, B, ldb, 1 - trans_b, f, s)) != ALP_OK) return st;
    double c = 0.0, r = 0.0;
    st = crt_choose_moduli(trans_a, trans_b, M, N, K, A, lda, B, ldb, e, f, ws + L0.off_g, s,
                           nmoduli, &c, &r);
    if (st == ALP_OK && predicted) {
        predicted[0] = c;
        predicted[1] = r;
    }
    return st;
}

alp_status alp_emul_tail_split(int tiles, int nslices, alp_slice_kind kind, int sms, int* n_full,
                               int* pieces, int* t_lo, int* t_hi) {
    EmulScheme sc;
    if (tiles < 0 || !emul_scheme_of(kind, &sc) || nslices < 1 ||
        nslices > (sc.crt ? kCrtMaxModuli : emul_max_slices(sc.b)) || sms < 1 || !n_full ||
        !pieces || !t_lo || !t_hi)
        return ALP_ERR_INVALID_ARG;
    const TailSplit ts = tail_split(tiles, nslices, sms, sc.trim, sc.crt);
    *n_full = ts.n_full;
    *pieces = ts.pieces;
    for (int i = 0; i < 8; ++i) {
        t_lo[i] = ts.t_lo[i];
        t_hi[i] = ts.t_hi[i];
    }
    return ALP_OK;
}

alp_status alp_emul_exponents(int64_t rows, int64_t cols, const double* X, int64_t ldx,
                              int trans, int32_t* exps, void* stream) {
    if (rows < 0 || cols < 0 || !exps || (rows > 0 && cols > 0 && !X)) return ALP_ERR_INVALID_ARG;
    if (rows == 0) return ALP_OK;
    if (!trans && ldx < cols) return ALP_ERR_INVALID_ARG;
    if (trans && ldx < rows) return ALP_ERR_INVALID_ARG;
    return emul_exponents(rows, cols, X, ldx, trans, exps, reinterpret_cast<cudaStream_t>(stream));
}

alp_status alp_emul_split(int64_t R, int64_t K, const double* X, int64_t ldx, int trans,
                          const int32_t* exps, int nslices, alp_slice_kind kind, void* out_bf16,
                          int64_t kpad, void* stream) {
    EmulScheme sc;
    if (R < 0 || K < 0 || !emul_scheme_of(kind, &sc) ||
        (sc.crt ? !emul_slices_ok(sc, nslices, false)
                : (nslices < 1 || nslices > emul_max_slices(sc.b))) ||
        kpad < K || kpad % 64 || !exps || !out_bf16 || (R > 0 && K > 0 && !X))
        return ALP_ERR_INVALID_ARG;
    if (!trans && ldx < K) return ALP_ERR_INVALID_ARG;
    if (trans && ldx < R) return ALP_ERR_INVALID_ARG;
    if (sc.crt && (K > kCrtMaxK || crt_bits(K, nslices) < 1)) return ALP_ERR_UNSUPPORTED;
    if (R == 0 || kpad == 0) return ALP_OK;
    if (sc.crt)
        return emul_split_crt(R, K, X, ldx, trans, exps, nslices,
                              reinterpret_cast<__nv_bfloat16*>(out_bf16), kpad,
                              crt_bits(K, nslices), reinterpret_cast<cudaStream_t>(stream));
    return emul_split(R, K, X, ldx, trans, exps, nslices,
                      reinterpret_cast<__nv_bfloat16*>(out_bf16), kpad,
                      reinterpret_cast<cudaStream_t>(stream), sc.b);
}

alp_status alp_emul_scan_split_rows(int64_t R, int64_t K, const double* X, int64_t ldx,
                                    int32_t* exps, int nslices, alp_slice_kind kind,
                                    void* out_bf16, int64_t kpad, void* stream) {
    EmulScheme sc;
    if (R < 0 || K < 0 || !emul_scheme_of(kind, &sc) || !sc.crt ||
        !emul_slices_ok(sc, nslices, false) || kpad < K || kpad % 64 || ldx < K || !exps ||
        !out_bf16 || (R > 0 && K > 0 && !X) || ((uintptr_t)out_bf16 & 7))
        return ALP_ERR_INVALID_ARG;
    if (K > kCrtMaxK || crt_bits(K, nslices) < 1) return ALP_ERR_UNSUPPORTED;
    if (R == 0) return ALP_OK;
    return emul_scan_split_crt(R, K, X, ldx, exps, nslices,
                               reinterpret_cast<__nv_bfloat16*>(out_bf16), kpad,
                               crt_bits(K, nslices), reinterpret_cast<cudaStream_t>(stream));
}

alp_status alp_emul_slice_products(int64_t M, int64_t N, int64_t K, int nslices,
                                   alp_slice_kind kind, const void* da_bf16, const void* db_bf16,
                                   int64_t kpad, void* G, int64_t ldg, void* stream) {
    EmulScheme sc;
    if (M < 0 || N < 0 || K < 0 || !emul_scheme_of(kind, &sc) ||
        (sc.crt ? !emul_slices_ok(sc, nslices, false)
                : (nslices < 1 || nslices > emul_max_slices(sc.b))) ||
        kpad < K || kpad % kEmulBK || ldg < N || ldg % 256 || K > emul_scheme_max_k(sc))
        return ALP_ERR_INVALID_ARG;
    if (M == 0 || N == 0 || K == 0) return ALP_OK;
    if (!da_bf16 || !db_bf16 || !G || ((uintptr_t)G & 15)) return ALP_ERR_INVALID_ARG;
    return emul_slice_gemm(M, N, K, nslices, reinterpret_cast<const __nv_bfloat16*>(da_bf16),
                           reinterpret_cast<const __nv_bfloat16*>(db_bf16), kpad,
                           static_cast<int32_t*>(G), ldg,
                           reinterpret_cast<cudaStream_t>(stream), 0, 0, sc.b, sc.trim, sc.crt);
}

alp_status alp_emul_recombine(int64_t M, int64_t N, int nslices, alp_slice_kind kind,
                              const int32_t* G, int64_t ldg, const int32_t* e, const int32_t* f,
                              double alpha, double beta, double* C, int64_t ldc, void* stream) {
    EmulScheme sc;
    if (M < 0 || N < 0 || !emul_scheme_of(kind, &sc) || sc.crt || nslices < 1 ||
        nslices > emul_max_slices(sc.b) || ldg < N || ldc < N)
        return ALP_ERR_INVALID_ARG;
    if (M == 0 || N == 0) return ALP_OK;
    if (!G || !e || !f || !C) return ALP_ERR_INVALID_ARG;
    return launch_recombine(nslices, sc.b, recombine_grid(M, N),
                            reinterpret_cast<cudaStream_t>(stream), G, M * ldg, ldg, e, f, M, N,
                            alpha, beta, C, ldc);
}

int alp_emul_crt_bits(int64_t K, int nmoduli) {
    if (K < 0 || nmoduli < kCrtMinModuli || nmoduli > kCrtMaxModuli || K > kCrtMaxK) return 0;
    return crt_bits(K, nmoduli);
}

alp_status alp_emul_recombine_crt(int64_t M, int64_t N, int64_t K, int nmoduli,
                                  const uint8_t* R, int64_t ldr, const int32_t* e,
                                  const int32_t* f, double alpha, double beta, double* C,
                                  int64_t ldc, void* stream) {
    if (M < 0 || N < 0 || K < 0 || nmoduli < kCrtMinModuli || nmoduli > kCrtMaxModuli ||
        ldr < N || ldc < N)
        return ALP_ERR_INVALID_ARG;
    const int k = alp_emul_crt_bits(K, nmoduli);
    if (k < 1) return ALP_ERR_UNSUPPORTED;
    if (M == 0 || N == 0) return ALP_OK;
    if (!R || !e || !f || !C) return ALP_ERR_INVALID_ARG;
    return launch_recombine_crt(nmoduli, k, recombine_grid(M, N),
                                reinterpret_cast<cudaStream_t>(stream), R, M * ldr, ldr, e, f, M,
                                N, alpha, beta, C, ldc);
}

size_t alp_emul_products_recombine_crt_workspace(int64_t M, int64_t N) {
    return emul_crt_sched_bytes(M, N);
}

alp_status alp_emul_products_recombine_crt(int64_t M, int64_t N, int64_t K, int nmoduli,
                                           const void* da_bf16, const void* db_bf16,
                                           int64_t kpad, uint8_t* R, int64_t ldr,
                                           const int32_t* e, const int32_t* f, double alpha,
                                           double beta, double* C, int64_t ldc, void* workspace,
                                           size_t workspace_bytes, void* stream) {
    if (M < 0 || N < 0 || K < 1 || nmoduli < kCrtMinModuli || nmoduli > kCrtMaxModuli ||
        kpad < K || kpad % kEmulBK || ldr < N || ldr % 256 || ldc < N || K > kCrtMaxK)
        return ALP_ERR_INVALID_ARG;
    const int k = alp_emul_crt_bits(K, nmoduli);
    if (k < 1) return ALP_ERR_UNSUPPORTED;
    if (M == 0 || N == 0) return ALP_OK;
    if (!da_bf16 || !db_bf16 || !R || ((uintptr_t)R & 15) || !e || !f || !C ||
        ((uintptr_t)C & 7))
        return ALP_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 3) ||
        workspace_bytes < emul_crt_sched_bytes(M, N))
        return ALP_ERR_WORKSPACE;
    return emul_crt_products_recombine(M, N, K, nmoduli,
                                       reinterpret_cast<const __nv_bfloat16*>(da_bf16),
                                       reinterpret_cast<const __nv_bfloat16*>(db_bf16), kpad, R,
                                       ldr, e, f, k, alpha, beta, C, ldc,
                                       static_cast<int*>(workspace), workspace_bytes,
                                       reinterpret_cast<cudaStream_t>(stream), 0, 0, 1);
}

alp_status alp_gemm_f64_emul(int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                             int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                             int64_t ldc, int nslices, alp_slice_kind kind, void* workspace,
                             size_t workspace_bytes, void* stream) {
    return emul_gemm_impl<double>(0, 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nslices,
                                  kind, workspace, workspace_bytes,
                                  reinterpret_cast<cudaStream_t>(stream));
}

alp_status alp_gemm_f64_emul_ex(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                                double alpha, const double* A, int64_t lda, const double* B,
                                int64_t ldb, double beta, double* C, int64_t ldc, int nslices,
                                alp_slice_kind kind, void* workspace, size_t workspace_bytes,
                                void* stream) {
    return emul_gemm_impl<double>(trans_a, trans_b, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                  nslices, kind, workspace, workspace_bytes,
                                  reinterpret_cast<cudaStream_t>(stream));
}

// ---- FP32 operands and results ----

size_t alp_gemm_f32_emul_workspace(int64_t M, int64_t N, int64_t K, int nslices,
                                   alp_slice_kind kind) {
    EmulScheme sc;
    if (M < 0 || N < 0 || K < 0 || !emul_scheme_of(kind, &sc) || !emul_slices_ok(sc, nslices, true))
        return 0;
    return emul_layout(M, N, K, nslices).bytes;
}

alp_status alp_emul_exponents_f32(int64_t rows, int64_t cols, const float* X, int64_t ldx,
                                  int trans, int32_t* exps, void* stream) {
    if (rows < 0 || cols < 0 || !exps || (rows > 0 && cols > 0 && !X)) return ALP_ERR_INVALID_ARG;
    if (rows == 0) return ALP_OK;
    if (!trans && ldx < cols) return ALP_ERR_INVALID_ARG;
    if (trans && ldx < rows) return ALP_ERR_INVALID_ARG;
    return emul_exponents(rows, cols, X, ldx, trans, exps, reinterpret_cast<cudaStream_t>(stream));
}

alp_status alp_emul_split_f32(int64_t R, int64_t K, const float* X, int64_t ldx, int trans,
                              const int32_t* exps, int nslices, alp_slice_kind kind,
                              void* out_bf16, int64_t kpad, void* stream) {
    EmulScheme sc;
    if (R < 0 || K < 0 || !emul_scheme_of(kind, &sc) || sc.crt || nslices < 1 ||
        nslices > emul_max_slices_f32(sc.b) || kpad < K || kpad % 64 || !exps || !out_bf16 ||
        (R > 0 && K > 0 && !X))
        return ALP_ERR_INVALID_ARG;
    if (!trans && ldx < K) return ALP_ERR_INVALID_ARG;
    if (trans && ldx < R) return ALP_ERR_INVALID_ARG;
    if (R == 0 || kpad == 0) return ALP_OK;
    return emul_split(R, K, X, ldx, trans, exps, nslices,
                      reinterpret_cast<__nv_bfloat16*>(out_bf16), kpad,
                      reinterpret_cast<cudaStream_t>(stream), sc.b);
}

alp_status alp_emul_recombine_f32(int64_t M, int64_t N, int nslices, alp_slice_kind kind,
                                  const int32_t* G, int64_t ldg, const int32_t* e,
                                  const int32_t* f, float alpha, float beta, float* C,
                                  int64_t ldc, void* stream) {
    EmulScheme sc;
    if (M < 0 || N < 0 || !emul_scheme_of(kind, &sc) || sc.crt || nslices < 1 ||
        nslices > emul_max_slices_f32(sc.b) || ldg < N || ldc < N)
        return ALP_ERR_INVALID_ARG;
    if (M == 0 || N == 0) return ALP_OK;
    if (!G || !e || !f || !C) return ALP_ERR_INVALID_ARG;
    return launch_recombine_f32(nslices, sc.b, recombine_grid(M, N),
                                reinterpret_cast<cudaStream_t>(stream), G, M * ldg, ldg, e, f, M,
                                N, alpha, beta, C, ldc);
}

alp_status alp_gemm_f32_emul(int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                             int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                             int64_t ldc, int nslices, alp_slice_kind kind, void* workspace,
                             size_t workspace_bytes, void* stream) {
    return emul_gemm_impl<float>(0, 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nslices,
                                 kind, workspace, workspace_bytes,
                                 reinterpret_cast<cudaStream_t>(stream));
}

alp_status alp_gemm_f32_emul_ex(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                                float alpha, const float* A, int64_t lda, const float* B,
                                int64_t ldb, float beta, float* C, int64_t ldc, int nslices,
                                alp_slice_kind kind, void* workspace, size_t workspace_bytes,
                                void* stream) {
    return emul_gemm_impl<float>(trans_a, trans_b, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                 nslices, kind, workspace, workspace_bytes,
                                 reinterpret_cast<cudaStream_t>(stream));
}

// ---- column-major calls: C^T = op(B)^T op(A)^T in row-major terms ----

size_t alp_gemm_f64_emul_cm_workspace(int64_t M, int64_t N, int64_t K, int nslices,
                                      alp_slice_kind kind) {
    return alp_gemm_f64_emul_workspace(N, M, K, nslices, kind);
}

alp_status alp_gemm_f64_emul_cm(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                                double alpha, const double* A, int64_t lda, const double* B,
                                int64_t ldb, double beta, double* C, int64_t ldc, int nslices,
                                alp_slice_kind kind, void* workspace, size_t workspace_bytes,
                                void* stream) {
    return emul_gemm_impl<double>(trans_b, trans_a, N, M, K, alpha, B, ldb, A, lda, beta, C, ldc,
                                  nslices, kind, workspace, workspace_bytes,
                                  reinterpret_cast<cudaStream_t>(stream));
}

size_t alp_gemm_f32_emul_cm_workspace(int64_t M, int64_t N, int64_t K, int nslices,
                                      alp_slice_kind kind) {
    return alp_gemm_f32_emul_workspace(N, M, K, nslices, kind);
}

alp_status alp_gemm_f32_emul_cm(int trans_a, int trans_b, int64_t M, int64_t N, int64_t K,
                                float alpha, const float* A, int64_t lda, const float* B,
                                int64_t ldb, float beta, float* C, int64_t ldc, int nslices,
                                alp_slice_kind kind, void* workspace, size_t workspace_bytes,
                                void* stream) {
    return emul_gemm_impl<float>(trans_b, trans_a, N, M, K, alpha, B, ldb, A, lda, beta, C, ldc,
                                 nslices, kind, workspace, workspace_bytes,
                                 reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
