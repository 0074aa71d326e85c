// The modular (Chinese remainder) variant of the emulated FP64 GEMM, after
// Ozaki, Uchino and Imamura's scheme II: each operand is rounded to k-bit
// integers per row (A) and column (B), A'_ik = RN(A_ik 2^(k - e_i)), and the
// exact integer product P = A' B' is obtained from its residues modulo n
// pairwise coprime moduli m_l <= 256: the residues of A' and B' (in
// [-128, 127], exact in bf16) are multiplied on the tensor cores by the
// slice-product kernel (one product per modulus instead of one per digit
// pair; the epilogue reduces each sum to a weighted residue byte), and P
// follows by the Chinese remainder theorem, exactly, because
// |P| <= K 2^(2k) < M / 2 with M = m_1 ... m_n.  C = alpha RN(P 2^(e_i + f_j
// - 2k)) (+ fma(beta, C, .)).
#include <cstdint>

#include "crt.cuh"
#include "emul.cuh"
#include "emul_split.cuh"

namespace alp {

// The largest k <= 60 with K 2^(2k+1) <= M (1 - 2^-18): then |P| <= K 2^(2k)
// stays below M / 2 by at least M 2^-19, more than the error of the
// reconstruction's fixed-point quotient (below 2^-21 in units of M), so that
// quotient rounds to the right multiple of M.
int crt_bits(int64_t K, int n) {
    if (n < 1 || n > kCrtMaxModuli) return 0;
    unsigned __int128 M = 1;
    for (int l = 0; l < n; ++l) M *= crt_modulus(l);
    const unsigned __int128 lim = M - (M >> 18);
    const uint64_t Kc = K > 0 ? (uint64_t)K : 1;
    int kbits = 0;
    while ((Kc >> kbits) != 0) ++kbits;
    for (int k = 60; k >= 1; --k) {
        const int sh = 2 * k + 1;
        if (sh + kbits > 127) continue;                      // K 2^sh > 2^126 > M
        if (((unsigned __int128)Kc << sh) <= lim) return k;
    }
    return 0;
}

uint32_t crt_weight(int n, int l) {
    if (n < 1 || n > kCrtMaxModuli || l < 0 || l >= n) return 0;
    const uint32_t m = crt_modulus(l);
    uint32_t r = 1;   // Mn / m_l mod m_l = prod_{i != l} m_i mod m_l
    for (int i = 0; i < n; ++i)
        if (i != l) r = (r * (crt_modulus(i) % m)) % m;
    for (uint32_t y = 1; y < m; ++y)
        if ((r * y) % m == 1u) return y;
    return 0;
}

// The splitter.  A' = RN(a 2^(k - e)) straight from the IEEE fields: a =
// +-mant 2^E, shifted left when sh = E + k - e >= 0 (exact; |A'| < 2^k since
// |a| < 2^e), else rounded half to even at bit -sh (0 below 2^-54 of mant).
// Then the signed A' = hi 2^40 + mid 2^20 + lo (hi signed, |hi| <= 2^20; mid,
// lo in [0, 2^20)) and per modulus x = hi (2^40 mod m) + mid (2^20 mod m) + lo
// + b_m with b_m = m ceil(2^28 / m) + floor(m / 2), so that 0 < x < 2^30 and
// x = A' + floor(m / 2) (mod m); the residue moved to [-floor(m/2),
// ceil(m/2)) is (x mod m) - floor(m / 2), whose subtraction folds into the
// bf16 packing.
__host__ __device__ constexpr uint32_t crt_split_bias(uint32_t m) {
    return m * (((1u << 28) + m - 1) / m) + m / 2;
}
struct CrtSplit {
    int k;
    template <int S>
    __device__ __forceinline__ void split(double a, int e, int (&d)[S]) const {
        const uint64_t bits = (uint64_t)__double_as_longlong(a);
        const int ex = (int)((bits >> 52) & 0x7FF);
        uint64_t mant = bits & ((1ull << 52) - 1);
        int E = -1074;
        if (ex == 0x7FF) mant = 0;   // Inf/NaN: reported by the scan; residues 0
        else if (ex) {
            mant |= 1ull << 52;
            E = ex - 1075;
        }
        const int sh = E + k - e;
        uint64_t u;
        if (sh >= 0) {
            u = mant << (sh > 63 ? 63 : sh);
        } else if (sh < -54) {
            u = 0;
        } else {
            const int r = -sh;
            const uint64_t q = mant >> r, rem = mant & ((1ull << r) - 1), half = 1ull << (r - 1);
            u = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
        }
        const int64_t v = (int64_t)bits < 0 ? -(int64_t)u : (int64_t)u;
        const int32_t hi = (int32_t)(v >> 40);
        const uint32_t mid = (uint32_t)(v >> 20) & 0xFFFFFu, lo = (uint32_t)v & 0xFFFFFu;
#pragma unroll
        for (int l = 0; l < S; ++l) {
            const uint32_t m = crt_modulus(l);
            const int32_t x = hi * (int32_t)crt_pow2_mod(40, m) +
                              (int32_t)(mid * crt_pow2_mod(20, m) + (lo + crt_split_bias(m)));
            d[l] = (int)crt_mod((uint32_t)x, m) - (int)(m / 2);
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
    // 128-thread blocks (4 k per thread), registers capped for 6 blocks per
    // SM (measured faster than 256 threads, and than the uncapped 100
    // registers)
    const int64_t bx = (kpad + 511) / 512;
    int64_t by = (int64_t)device_sm_count() * 16 / bx;
    by = by < 1 ? 1 : by > R ? R : by > 65535 ? 65535 : by;
    const dim3 grid4((unsigned)bx, (unsigned)by);
    int64_t blocks = (R * (kpad / 2) + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    blocks = blocks > cap ? cap : blocks < 1 ? 1 : blocks;
#define ALP_CRT_SPLIT_CASE(x)                                                                    \
    case x:                                                                                      \
        if (!trans && vec)                                                                       \
            split_rows4_kernel<T, x, CrtSplit, 128, 6><<<grid4, 128, 0, st>>>(X, R, K, ldx, exps, \
                                                                              out, kpad, sp);     \
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

// Chinese remainder reconstruction constants for n moduli: Mn = prod m_l and
// M_l = Mn / m_l as four 32-bit limbs, and F_l = round(2^32 / m_l).
struct CrtRecConsts {
    uint32_t ml[kCrtMaxModuli][4];
    uint32_t mn[4];
    uint32_t F[kCrtMaxModuli];
    int k;
};

static CrtRecConsts crt_consts(int n, int k) {
    CrtRecConsts c{};
    unsigned __int128 M = 1;
    for (int l = 0; l < n; ++l) M *= crt_modulus(l);
    for (int i = 0; i < 4; ++i) c.mn[i] = (uint32_t)(M >> (32 * i));
    for (int l = 0; l < n; ++l) {
        const uint32_t m = crt_modulus(l);
        const unsigned __int128 Ml = M / m;
        for (int i = 0; i < 4; ++i) c.ml[l][i] = (uint32_t)(Ml >> (32 * i));
        c.F[l] = (uint32_t)(((1ull << 32) + m / 2) / m);
    }
    c.k = k;
    return c;
}

__device__ __forceinline__ uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c) {
    uint64_t d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// Four columns per thread: the n bytes x_l = (P y_l) mod m_l (four adjacent
// columns in one 32-bit load per plane) give sum_l x_l M_l = P + c Mn for the
// integer c = round(sum_l x_l / m_l) (|P| / Mn <= 1/2 - 2^-19).  The sum is
// kept as four 64-bit column sums of 32-bit limbs (each below 16 * 2^8 *
// 2^32), c from a 32.32 fixed-point sum whose error is below 2^-21, and P =
// sum - c Mn follows by one carry pass, exact modulo 2^128, which holds it.
template <int S>
__global__ void __launch_bounds__(128) recombine_crt_kernel(
    const uint8_t* __restrict__ R, int64_t rplane, int64_t ldr, const int32_t* __restrict__ e,
    const int32_t* __restrict__ f, int64_t M, int64_t N, double alpha, double beta,
    double* __restrict__ C, int64_t ldc, bool rvec, const CrtRecConsts cc) {
    for (int64_t i = blockIdx.y; i < M; i += gridDim.y) {
        const int ei = e[i] - 2 * cc.k;
        const uint8_t* ri = R + i * ldr;
        double* ci = C + i * ldc;
        const bool cvec = (reinterpret_cast<uintptr_t>(ci) & 15) == 0;
        for (int64_t j = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); j < N;
             j += 4 * (int64_t)gridDim.x * blockDim.x) {
            uint32_t v[S];
#pragma unroll
            for (int t = 0; t < S; ++t) {
                const uint8_t* g = ri + (int64_t)t * rplane + j;
                if (rvec) {   // ldr and j are multiples of 4: the word stays in the row
                    v[t] = __ldg(reinterpret_cast<const uint32_t*>(g));
                } else {
                    v[t] = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (j + b < N) v[t] |= (uint32_t)__ldg(g + b) << (8 * b);
                }
            }
            // two columns at a time (two independent chains), byte u of each
            // plane word by one byte permute
            double o[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 1
            for (int up = 0; up < 2; ++up) {
                if (j + 2 * up >= N) break;
                const uint32_t s0 = 0x4440u + 2u * (uint32_t)up, s1 = s0 + 1u;
                uint64_t a[2][4] = {}, qa[2] = {};
#pragma unroll
                for (int t = 0; t < S; ++t) {
                    const uint32_t x0 = __byte_perm(v[t], 0u, s0), x1 = __byte_perm(v[t], 0u, s1);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        a[0][q] = mad_wide(x0, cc.ml[t][q], a[0][q]);
                        a[1][q] = mad_wide(x1, cc.ml[t][q], a[1][q]);
                    }
                    qa[0] = mad_wide(x0, cc.F[t], qa[0]);
                    qa[1] = mad_wide(x1, cc.F[t], qa[1]);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t jj = j + 2 * up + h;
                    const uint32_t qi = (uint32_t)((qa[h] + 0x80000000ull) >> 32);
                    int64_t c = (int64_t)a[h][0] - (int64_t)((uint64_t)qi * cc.mn[0]);
                    const uint32_t w0 = (uint32_t)c;
                    c = (c >> 32) + (int64_t)a[h][1] - (int64_t)((uint64_t)qi * cc.mn[1]);
                    const uint32_t w1 = (uint32_t)c;
                    c = (c >> 32) + (int64_t)a[h][2] - (int64_t)((uint64_t)qi * cc.mn[2]);
                    const uint32_t w2 = (uint32_t)c;
                    c = (c >> 32) + (int64_t)a[h][3] - (int64_t)((uint64_t)qi * cc.mn[3]);
                    const uint32_t w3 = (uint32_t)c;
                    const int64_t hi = (int64_t)(((uint64_t)w3 << 32) | w2);
                    const uint64_t lo = ((uint64_t)w1 << 32) | w0;
                    // a column past N computes from the row's padding and is not stored
                    const double w = i128_scaled_to_double_rn(hi, lo, ei + (jj < N ? __ldg(f + jj) : 0));
                    double out = (alpha == 1.0) ? w : (alpha == -1.0) ? -w : alpha * w;
                    if (beta != 0.0 && jj < N) out = __fma_rn(beta, ci[jj], out);
                    if (up == 0) {
                        if (h == 0) o[0] = out; else o[1] = out;
                    } else {
                        if (h == 0) o[2] = out; else o[3] = out;
                    }
                }
            }
            if (cvec && j + 3 < N) {
                reinterpret_cast<double2*>(ci + j)[0] = make_double2(o[0], o[1]);
                reinterpret_cast<double2*>(ci + j)[1] = make_double2(o[2], o[3]);
            } else {
                ci[j] = o[0];
                if (j + 1 < N) ci[j + 1] = o[1];
                if (j + 2 < N) ci[j + 2] = o[2];
                if (j + 3 < N) ci[j + 3] = o[3];
            }
        }
    }
}

alp_status launch_recombine_crt(int n, int k, dim3 grid, cudaStream_t st, const uint8_t* R,
                                int64_t rplane, int64_t ldr, const int32_t* e, const int32_t* f,
                                int64_t M, int64_t N, double alpha, double beta, double* C,
                                int64_t ldc) {
    if (k < 1 || k > 60) return ALP_ERR_UNSUPPORTED;
    const CrtRecConsts cc = crt_consts(n, k);
    const bool rvec = (reinterpret_cast<uintptr_t>(R) & 3) == 0 && rplane % 4 == 0 && ldr % 4 == 0;
    // four columns per thread, 128-thread blocks: 512 columns per block, as
    // the grid was sized
#define ALP_CRT_REC_CASE(x)                                                                       \
    case x:                                                                                      \
        recombine_crt_kernel<x><<<grid, 128, 0, st>>>(R, rplane, ldr, e, f, M, N, alpha, beta, C, \
                                                      ldc, rvec, cc);                            \
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
