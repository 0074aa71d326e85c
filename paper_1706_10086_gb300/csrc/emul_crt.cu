// The modular (Chinese remainder) variant of the emulated FP64 GEMM, after
// Ozaki, Uchino and Imamura's scheme II: each operand is rounded to k-bit
// integers per row (A) and column (B), A'_ik = RN(A_ik 2^(k - e_i)), and the
// exact integer product P = A' B' is obtained from its residues modulo n
// pairwise coprime moduli m_l <= 256: the residues of A' and B' (in
// [-128, 127], exact in bf16) are multiplied on the tensor cores by the
// slice-product kernel (one product per modulus instead of one per digit
// pair), and P follows by the Chinese remainder theorem, exactly, because
// |P| <= K 2^(2k) <= M / 4 with M = m_1 ... m_n.  C = alpha RN(P 2^(e_i + f_j
// - 2k)) (+ fma(beta, C, .)).
#include <cstdint>

#include "emul.cuh"
#include "emul_split.cuh"

namespace alp {

// The moduli, largest first (pairwise coprime; 256 = 2^8 first).
__host__ __device__ __forceinline__ constexpr uint32_t crt_modulus(int l) {
    switch (l) {
        case 0: return 256u;
        case 1: return 255u;
        case 2: return 253u;
        case 3: return 251u;
        case 4: return 247u;
        case 5: return 241u;
        case 6: return 239u;
        case 7: return 233u;
        case 8: return 229u;
        case 9: return 227u;
        case 10: return 223u;
        case 11: return 217u;
        case 12: return 211u;
        case 13: return 199u;
        case 14: return 197u;
        case 15: return 193u;
        default: return 1u;
    }
}
// 2^bits mod m.
__host__ __device__ __forceinline__ constexpr uint32_t crt_pow2_mod(int bits, uint32_t m) {
    uint32_t r = 1u % m;
    for (int i = 0; i < bits; ++i) r = (r * 2u) % m;
    return r;
}
// x mod m for x < 2^30: q = floor(x ceil(2^38 / m) / 2^38) is exact for m <= 255
// (the product over-estimates x / m by less than 2^-8, and x mod m <= m - 1
// keeps the fraction below 1 - 1/m); m = 256 is a mask.
__device__ __forceinline__ uint32_t crt_mod(uint32_t x, uint32_t m) {
    if (m == 256u) return x & 255u;
    const uint32_t magic = (uint32_t)(((1ull << 38) + m - 1) / m);
    return x - (__umulhi(x, magic) >> 6) * m;
}

// P must satisfy K 2^(2k + 2) <= M (so |P| <= M / 4); the largest such k <= 60.
int crt_bits(int64_t K, int n) {
    if (n < 1 || n > kCrtMaxModuli) return 0;
    unsigned __int128 M = 1;
    for (int l = 0; l < n; ++l) M *= crt_modulus(l);
    const uint64_t Kc = K > 0 ? (uint64_t)K : 1;
    int kbits = 0;
    while ((Kc >> kbits) != 0) ++kbits;
    for (int k = 60; k >= 1; --k) {
        const int sh = 2 * k + 2;
        if (sh + kbits > 127) continue;                      // K 2^sh > 2^126 > M
        if (((unsigned __int128)Kc << sh) <= M) return k;
    }
    return 0;
}

// The splitter: A' = RN(a 2^(k - e)) from the rounded-to-odd fixed point (the
// rounding sits at least 2 bits above its sticky bit, so it is exact), then
// |A'| = hi 2^40 + mid 2^20 + lo, and per modulus x = hi (2^40 mod m) + mid
// (2^20 mod m) + lo < 2^30, r = x mod m, negated for A' < 0, and moved to
// [-m/2, m/2).
struct CrtSplit {
    int k;
    template <int S>
    __device__ __forceinline__ void split(double a, int e, int (&d)[S]) const {
        const uint64_t X = fixed_point_r0(a, e);
        const int SH = 62 - k;
        const uint64_t odd = (X >> SH) & 1;
        const int64_t v = (int64_t)(X + ((1ull << (SH - 1)) - 1) + odd) >> SH;
        const bool neg = v < 0;
        const uint64_t u = neg ? (uint64_t)(-v) : (uint64_t)v;
        const uint32_t lo = (uint32_t)(u & 0xFFFFFu), mid = (uint32_t)((u >> 20) & 0xFFFFFu);
        const uint32_t hi = (uint32_t)(u >> 40);
#pragma unroll
        for (int l = 0; l < S; ++l) {
            const uint32_t m = crt_modulus(l);
            const uint32_t x = hi * crt_pow2_mod(40, m) + mid * crt_pow2_mod(20, m) + lo;
            uint32_t r = crt_mod(x, m);
            if (neg && r) r = m - r;
            d[l] = (2u * r >= m + (m & 1u)) ? (int)r - (int)m : (int)r;
        }
    }
};

template <typename T>
alp_status emul_split_crt(int64_t R, int64_t K, const T* X, int64_t ldx, int trans,
                          const int32_t* exps, int n, __nv_bfloat16* out, int64_t kpad, int k,
                          cudaStream_t st) {
    if (k < 1 || k > 60) return ALP_ERR_UNSUPPORTED;
    const CrtSplit sp{k};
    const bool vec = (reinterpret_cast<uintptr_t>(out) & 7) == 0 && kpad % 4 == 0;
    const int64_t bx = (kpad + 1023) / 1024;
    int64_t by = (int64_t)device_sm_count() * 8 / bx;
    by = by < 1 ? 1 : by > R ? R : by > 65535 ? 65535 : by;
    const dim3 grid4((unsigned)bx, (unsigned)by);
    int64_t blocks = (R * (kpad / 2) + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    blocks = blocks > cap ? cap : blocks < 1 ? 1 : blocks;
#define ALP_CRT_SPLIT_CASE(x)                                                                    \
    case x:                                                                                      \
        if (!trans && vec)                                                                       \
            split_rows4_kernel<T, x, CrtSplit><<<grid4, 256, 0, st>>>(X, R, K, ldx, exps, out,    \
                                                                      kpad, sp);                  \
        else if (!trans)                                                                         \
            split_rows_kernel<T, x, CrtSplit><<<(unsigned)blocks, 256, 0, st>>>(                  \
                X, R, K, ldx, exps, out, kpad, sp);                                              \
        else                                                                                     \
            split_cols_kernel<T, x, CrtSplit><<<dim3((unsigned)((R + 31) / 32),                   \
                                                     (unsigned)(kpad / 64)),                     \
                                                256, 0, st>>>(X, K, R, ldx, exps, out, kpad, sp); \
        break;
    switch (n) {
        ALP_CRT_SPLIT_CASE(4) ALP_CRT_SPLIT_CASE(5) ALP_CRT_SPLIT_CASE(6) ALP_CRT_SPLIT_CASE(7)
        ALP_CRT_SPLIT_CASE(8) ALP_CRT_SPLIT_CASE(9) ALP_CRT_SPLIT_CASE(10) ALP_CRT_SPLIT_CASE(11)
        ALP_CRT_SPLIT_CASE(12) ALP_CRT_SPLIT_CASE(13) ALP_CRT_SPLIT_CASE(14) ALP_CRT_SPLIT_CASE(15)
        ALP_CRT_SPLIT_CASE(16)
        default: return ALP_ERR_INVALID_ARG;
    }
#undef ALP_CRT_SPLIT_CASE
    return cuda_status(cudaGetLastError());
}
template alp_status emul_split_crt<double>(int64_t, int64_t, const double*, int64_t, int,
                                           const int32_t*, int, __nv_bfloat16*, int64_t, int,
                                           cudaStream_t);

// Chinese remainder reconstruction constants for n moduli: M = prod m_l,
// M_l = M / m_l (two 64-bit limbs), y_l = (M_l mod m_l)^-1 mod m_l, 1 / m_l.
struct CrtRecConsts {
    uint64_t ml_lo[kCrtMaxModuli], ml_hi[kCrtMaxModuli];
    uint64_t mm_lo, mm_hi;
    uint32_t y[kCrtMaxModuli];
    float inv[kCrtMaxModuli];
    int k;
};

static CrtRecConsts crt_consts(int n, int k) {
    CrtRecConsts c{};
    unsigned __int128 M = 1;
    for (int l = 0; l < n; ++l) M *= crt_modulus(l);
    c.mm_lo = (uint64_t)M;
    c.mm_hi = (uint64_t)(M >> 64);
    for (int l = 0; l < n; ++l) {
        const uint32_t m = crt_modulus(l);
        const unsigned __int128 Ml = M / m;
        c.ml_lo[l] = (uint64_t)Ml;
        c.ml_hi[l] = (uint64_t)(Ml >> 64);
        const uint32_t r = (uint32_t)(Ml % m);
        uint32_t y = 0;
        for (uint32_t t = 1; t < m; ++t)
            if ((r * t) % m == 1u) { y = t; break; }
        c.y[l] = y;
        c.inv[l] = 1.0f / (float)m;
    }
    c.k = k;
    return c;
}

// acc += x * (hi:lo) for a small x, modulo 2^128.
__device__ __forceinline__ void mad_u128(uint64_t& acc_lo, uint64_t& acc_hi, uint32_t x,
                                         uint64_t lo, uint64_t hi) {
    const uint64_t p_lo = lo * x, p_mid = __umul64hi(lo, x), p_hi = hi * x + p_mid;
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;"
        : "+l"(acc_lo), "+l"(acc_hi)
        : "l"(p_lo), "l"(p_hi));
}

// Four columns per thread as the digit-scheme recombination: the n group
// sums Q_l (int32, Q_l = P mod m_l up to multiples of m_l) of four adjacent
// columns arrive as one 16-byte load per plane.
template <int S>
__global__ void __launch_bounds__(256) recombine_crt_kernel(
    const int32_t* __restrict__ G, int64_t gplane, int64_t ldg, const int32_t* __restrict__ e,
    const int32_t* __restrict__ f, int64_t M, int64_t N, double alpha, double beta,
    double* __restrict__ C, int64_t ldc, bool gvec, const CrtRecConsts cc) {
    for (int64_t i = blockIdx.y; i < M; i += gridDim.y) {
        const int ei = e[i] - 2 * cc.k;
        const int32_t* gi = G + i * ldg;
        double* ci = C + i * ldc;
        const bool cvec = (reinterpret_cast<uintptr_t>(ci) & 15) == 0;
        for (int64_t j = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); j < N;
             j += 4 * (int64_t)gridDim.x * blockDim.x) {
            int4 v[S];
#pragma unroll
            for (int t = 0; t < S; ++t) {
                const int32_t* g = gi + (int64_t)t * gplane + j;
                if (gvec) v[t] = __ldg(reinterpret_cast<const int4*>(g));
                else v[t] = make_int4(__ldg(g), __ldg(g + 1), __ldg(g + 2), __ldg(g + 3));
            }
            double out[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (j + u >= N) break;
                uint64_t lo = 0, hi = 0;
                float q = 0.0f;
#pragma unroll
                for (int t = 0; t < S; ++t) {
                    const int32_t Q = u == 0 ? v[t].x : u == 1 ? v[t].y : u == 2 ? v[t].z : v[t].w;
                    const uint32_t m = crt_modulus(t);
                    uint32_t r = crt_mod(Q < 0 ? (uint32_t)(-(int64_t)Q) : (uint32_t)Q, m);
                    if (Q < 0 && r) r = m - r;
                    const uint32_t x = crt_mod(r * cc.y[t], m);
                    mad_u128(lo, hi, x, cc.ml_lo[t], cc.ml_hi[t]);
                    q = __fmaf_rn((float)x, cc.inv[t], q);
                }
                // sum x_l M_l = M (q_int + P / M) with |P| / M <= 1/4: subtract M rint(q)
                const uint32_t qi = (uint32_t)__float2int_rn(q);
                uint64_t s_lo = 0, s_hi = 0;
                mad_u128(s_lo, s_hi, qi, cc.mm_lo, cc.mm_hi);
                asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;"
                    : "+l"(lo), "+l"(hi)
                    : "l"(s_lo), "l"(s_hi));
                const double w = i128_scaled_to_double_rn((int64_t)hi, lo, ei + __ldg(f + j + u));
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

alp_status launch_recombine_crt(int n, int k, dim3 grid, cudaStream_t st, const int32_t* G,
                                int64_t gplane, int64_t ldg, const int32_t* e, const int32_t* f,
                                int64_t M, int64_t N, double alpha, double beta, double* C,
                                int64_t ldc) {
    if (k < 1 || k > 60) return ALP_ERR_UNSUPPORTED;
    const CrtRecConsts cc = crt_consts(n, k);
    const bool gvec = (reinterpret_cast<uintptr_t>(G) & 15) == 0 && gplane % 4 == 0 && ldg % 4 == 0;
    grid.x = (unsigned)((grid.x + 1) / 2);   // four columns per thread
#define ALP_CRT_REC_CASE(x)                                                                       \
    case x:                                                                                      \
        recombine_crt_kernel<x><<<grid, 256, 0, st>>>(G, gplane, ldg, e, f, M, N, alpha, beta, C, \
                                                      ldc, gvec, cc);                            \
        break;
    switch (n) {
        ALP_CRT_REC_CASE(4) ALP_CRT_REC_CASE(5) ALP_CRT_REC_CASE(6) ALP_CRT_REC_CASE(7)
        ALP_CRT_REC_CASE(8) ALP_CRT_REC_CASE(9) ALP_CRT_REC_CASE(10) ALP_CRT_REC_CASE(11)
        ALP_CRT_REC_CASE(12) ALP_CRT_REC_CASE(13) ALP_CRT_REC_CASE(14) ALP_CRT_REC_CASE(15)
        ALP_CRT_REC_CASE(16)
        default: return ALP_ERR_INVALID_ARG;
    }
#undef ALP_CRT_REC_CASE
    return cuda_status(cudaGetLastError());
}

}  // namespace alp
