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
#include "crt_rec.cuh"
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

// The splitter.  A' = RN(a 2^(k - e)): for k <= 51 (and a normal power of two
// 2^(k - e)) by one FP64 fma, else straight from the IEEE fields: a =
// +-mant 2^E, shifted left when sh = E + k - e >= 0 (exact; |A'| <= 2^k since
// |a| < 2^e), else rounded half to even at bit -sh (0 below 2^-54 of mant).
// The residues, written as the bf16 encodings of integers r = A' (mod m)
// with |r| <= 128 (the tensor-core stage's exactness bound):
//  * for k <= 51 (|A'| <= 2^51) in f32 arithmetic: A' = c3 2^39 + c2 2^26 +
//    c1 2^13 + c0 (c3 signed, |c3| <= 2^12; c2, c1, c0 in [0, 2^13)), each
//    chunk turned into a float through its encoding (no conversion
//    instruction), and per modulus x = c3 (2^39 mod m) + c2 (2^26 mod m) +
//    c1 (2^13 mod m) + c0 by three fmas, exact (|x| < 2^23); q = x * RN(1/m)
//    rounded to an integer through 1.5 2^23, and r = x - q m by one fma,
//    exact: q is RN(x / m) or one off it when x / m lies within 0.003 of a
//    half-integer, so |r| <= m / 2 + 0.7, an integer at most 128;
//  * otherwise in integers: A' = hi 2^40 + mid 2^20 + lo (hi signed, |hi| <=
//    2^20; mid, lo in [0, 2^20)) and x = hi (2^40 mod m) + mid (2^20 mod m) +
//    lo + b_m with b_m = m ceil(2^28 / m) + floor(m / 2), so that 0 < x < 2^30
//    and x = A' + floor(m / 2) (mod m); r = (x mod m) - floor(m / 2) in
//    [-floor(m/2), ceil(m/2)).
// A float holding an integer of at most 8 significant bits has that
// integer's bf16 encoding in its upper 16 bits, so packing two residues is
// one byte permutation.
__host__ __device__ constexpr uint32_t crt_split_bias(uint32_t m) {
    return m * (((1u << 28) + m - 1) / m) + m / 2;
}
// The f32 path's constants per modulus l: 2^13, 2^26, 2^39 mod m_l, RN(1/m_l)
// and m_l, read from the constant bank as fma operands.
struct CrtSplitF32 {
    float p13[kCrtMaxModuli], p26[kCrtMaxModuli], p39[kCrtMaxModuli], inv[kCrtMaxModuli],
        m[kCrtMaxModuli];
};
constexpr CrtSplitF32 make_crt_split_f32() {
    CrtSplitF32 c{};
    for (int l = 0; l < kCrtMaxModuli; ++l) {
        const uint32_t m = crt_modulus(l);
        c.p13[l] = (float)crt_pow2_mod(13, m);
        c.p26[l] = (float)crt_pow2_mod(26, m);
        c.p39[l] = (float)crt_pow2_mod(39, m);
        c.inv[l] = 1.0f / (float)m;
        c.m[l] = (float)m;
    }
    return c;
}
__constant__ CrtSplitF32 c_crt_split_f32 = make_crt_split_f32();

struct CrtSplit {
    int k;
    template <int S>
    __device__ __forceinline__ void split(double a, int e, int (&d)[S]) const {
        const uint64_t bits = (uint64_t)__double_as_longlong(a);
        const int ex = (int)((bits >> 52) & 0x7FF);
        const int se = k - e;
        if (k <= 51 && se >= -1022 && se <= 1023) {
            // a 2^se is exact (a scaling by a normal power of two; a result
            // below the normal range is below 1/2 in magnitude), so one fma
            // with 1.5 2^52 rounds it to the nearest integer, ties to even:
            // |a 2^se| <= 2^51 keeps the sum in [2^52, 2^53], where the
            // encoding grows by one per unit, and the difference of the two
            // encodings is the integer
            const double y =
                __fma_rn(a, __longlong_as_double((long long)(se + 1023) << 52), 6755399441055744.0);
            const int64_t v =
                ex == 0x7FF ? 0 : (int64_t)__double_as_longlong(y) - 0x4338000000000000ll;
            const uint32_t vl = (uint32_t)v, vh = (uint32_t)((uint64_t)v >> 32);
            const float f0 = __int_as_float(0x4B000000 | (vl & 0x1FFFu)) - 8388608.0f;
            const float f1 = __int_as_float(0x4B000000 | ((vl >> 13) & 0x1FFFu)) - 8388608.0f;
            const float f2 = __int_as_float(0x4B000000 | (__funnelshift_r(vl, vh, 26) & 0x1FFFu)) -
                             8388608.0f;
            const float f3 = __int_as_float(0x4B400000 + ((int32_t)vh >> 7)) - 12582912.0f;
            const CrtSplitF32& c = c_crt_split_f32;
#pragma unroll
            for (int l = 0; l < S; ++l) {
                const float x =
                    __fmaf_rn(f3, c.p39[l], __fmaf_rn(f2, c.p26[l], __fmaf_rn(f1, c.p13[l], f0)));
                const float q = __fadd_rn(__fmaf_rn(x, c.inv[l], 12582912.0f), -12582912.0f);
                d[l] = __float_as_int(__fmaf_rn(-q, c.m[l], x));
            }
            return;
        }
        uint64_t mant = bits & ((1ull << 52) - 1);
        int E = -1074;
        if (ex == 0x7FF) mant = 0;   // Inf/NaN: reported by the scan; residues 0
        else if (ex) {
            mant |= 1ull << 52;
            E = ex - 1075;
        }
        const int sh = E + se;
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
            const int r = (int)crt_mod((uint32_t)x, m) - (int)(m / 2);
            d[l] = __float_as_int(__int_as_float(0x4B400000 + r) - 12582912.0f);
        }
    }
    // two residues (float encodings) as packed bf16
    __device__ __forceinline__ uint32_t pack(int lo, int hi) const {
        return __byte_perm((uint32_t)lo, (uint32_t)hi, 0x7632);
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
    // SM (measured faster than 256 threads, than 5 blocks and than 2 k per
    // thread at 8 blocks)
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
        else if (vec)                                                                            \
            split_cols4_kernel<T, x, CrtSplit><<<dim3((unsigned)((R + 31) / 32),                  \
                                                      (unsigned)((kpad + 127) / 128)),           \
                                                 256, 0, st>>>(X, K, R, ldx, exps, out, kpad, sp); \
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
alp_status emul_scan_split_crt(int64_t R, int64_t K, const double* X, int64_t ldx,
                               int32_t* exps, int n, __nv_bfloat16* out, int64_t kpad, int k,
                               cudaStream_t st) {
    if (k < 1 || k > 60) return ALP_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(out) & 7) != 0 || kpad % 4 != 0) return ALP_ERR_INVALID_ARG;
    const CrtSplit sp{k};
    int64_t blocks = (int64_t)device_sm_count() * 6 * 4;   // rows walked by the blocks
    blocks = blocks > R ? R : blocks < 1 ? 1 : blocks;
    int* err = device_error_word();
#define ALP_CRT_SCAN_SPLIT_CASE(x)                                                            \
    case x:                                                                                  \
        scan_split_rows4_kernel<x, CrtSplit, 128, 6>                                         \
            <<<(unsigned)blocks, 128, 0, st>>>(X, R, K, ldx, exps, out, kpad, sp, err);      \
        break;
    switch (n) {
        ALP_CRT_SCAN_SPLIT_CASE(4) ALP_CRT_SCAN_SPLIT_CASE(5) ALP_CRT_SCAN_SPLIT_CASE(6)
        ALP_CRT_SCAN_SPLIT_CASE(7) ALP_CRT_SCAN_SPLIT_CASE(8) ALP_CRT_SCAN_SPLIT_CASE(9)
        ALP_CRT_SCAN_SPLIT_CASE(10) ALP_CRT_SCAN_SPLIT_CASE(11) ALP_CRT_SCAN_SPLIT_CASE(12)
        ALP_CRT_SCAN_SPLIT_CASE(13) ALP_CRT_SCAN_SPLIT_CASE(14) ALP_CRT_SCAN_SPLIT_CASE(15)
        ALP_CRT_SCAN_SPLIT_CASE(16)
        default: return ALP_ERR_INVALID_ARG;
    }
#undef ALP_CRT_SCAN_SPLIT_CASE
    return cuda_status(cudaGetLastError());
}

template alp_status emul_split_crt<double>(int64_t, int64_t, const double*, int64_t, int,
                                           const int32_t*, int, __nv_bfloat16*, int64_t, int,
                                           cudaStream_t);

CrtRecConsts crt_rec_consts(int n, int k) {
    CrtRecConsts c{};
    unsigned __int128 M = 1;
    for (int l = 0; l < n; ++l) M *= crt_modulus(l);
    for (int i = 0; i < 4; ++i) c.mn[i] = (uint32_t)(M >> (32 * i));
    for (int g = 0; 3 * g < n && g < kCrtMaxGroups; ++g) {
        uint32_t mg = 1;
        for (int l = 3 * g; l < 3 * g + 3 && l < n; ++l) mg *= crt_modulus(l);
        const unsigned __int128 Mg = M / mg;
        for (int i = 0; i < 4; ++i) c.mg[g][i] = (uint32_t)(Mg >> (32 * i));
        const uint64_t F = (uint64_t)(((unsigned __int128)1 << 58) + mg / 2) / mg;
        c.fg_lo[g] = (uint32_t)F;
        c.fg_hi[g] = (uint32_t)(F >> 32);
        for (int l = 3 * g; l < 3 * g + 3 && l < n; ++l) c.cl[l] = mg / crt_modulus(l);
    }
    c.n = n;
    c.k = k;
    return c;
}

// Four columns per thread: the n bytes of four adjacent columns arrive in one
// 32-bit load per plane (crt_rec.cuh for the arithmetic); one rounding to
// double per element, then alpha (amode 0: 1, 1: -1, 2: any) and the fused
// beta term (bmode 1), decided on the host so that the loop holds no FP64
// comparison.
template <int S>
__global__ void __launch_bounds__(128, 5) recombine_crt_kernel(
    const uint8_t* __restrict__ R, int64_t rplane, int64_t ldr, const int32_t* __restrict__ e,
    const int32_t* __restrict__ f, int64_t M, int64_t N, double alpha, double beta,
    double* __restrict__ C, int64_t ldc, bool rvec, int amode, int bmode,
    const CrtRecConsts cc) {
    for (int64_t i = blockIdx.y; i < M; i += gridDim.y) {
        const int ei = e[i] - 2 * cc.k;
        const uint8_t* ri = R + i * ldr;
        double* ci = C + i * ldc;
        const bool cvec = (reinterpret_cast<uintptr_t>(ci) & 15) == 0;
        for (int64_t j = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); j < N;
             j += 4 * (int64_t)gridDim.x * blockDim.x) {
            const bool full = j + 3 < N;
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
            int64_t hi[4];
            uint64_t lo[4];
            crt_reconstruct4<S>(v, cc, hi, lo);
            int fj[4];
            if (full) {
#pragma unroll
                for (int u = 0; u < 4; ++u) fj[u] = __ldg(f + j + u);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) fj[u] = j + u < N ? __ldg(f + j + u) : 0;
            }
            double o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                // a column past N computes from the row's padding and is not stored
                const double w = i128_scaled_to_double_rn(hi[u], lo[u], ei + fj[u]);
                o[u] = amode == 0 ? w : amode == 1 ? -w : alpha * w;
            }
            if (bmode) {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (full || j + u < N) o[u] = __fma_rn(beta, ci[j + u], o[u]);
            }
            if (cvec && full) {
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

// The same reconstruction with the residue rows staged in shared memory: a
// block keeps 512 columns (four per thread) and walks its rows, thread 0
// prefetching kCrtRecSlots rows ahead by bulk copies (one per plane, 512 bytes
// or the row's 16-byte-rounded tail), so that the loads of later rows overlap
// the arithmetic of this one.  Needs R, the plane stride and the row stride
// 16-byte aligned (the copies may read up to 15 padding bytes of a row past N).
// Every thread waits for its row's slot (bounded); one block barrier per row
// then agrees on success and frees the slot for its refill.
constexpr int kCrtRecSlots = 4;

template <int S>
__global__ void __launch_bounds__(128, 5) recombine_crt_staged_kernel(
    const uint8_t* __restrict__ R, int64_t rplane, int64_t ldr, const int32_t* __restrict__ e,
    const int32_t* __restrict__ f, int64_t M, int64_t N, double alpha, double beta,
    double* __restrict__ C, int64_t ldc, int amode, int bmode, const CrtRecConsts cc,
    uint64_t tmo, int* err) {
    __shared__ __align__(16) uint8_t slots[kCrtRecSlots][S][512];
    __shared__ uint64_t full[kCrtRecSlots];
    const int64_t j0 = (int64_t)blockIdx.x * 512;
    const int64_t jt = j0 + 4 * threadIdx.x;
    const uint32_t cb = (uint32_t)((N - j0 >= 512 ? 512 : ((N - j0) + 15) / 16 * 16));
    // rows of this block: blockIdx.y, blockIdx.y + gridDim.y, ...
    const int64_t nrows = M > blockIdx.y ? (M - blockIdx.y + gridDim.y - 1) / gridDim.y : 0;
    auto row_of = [&](int64_t r) { return (int64_t)blockIdx.y + r * gridDim.y; };
    auto issue = [&](int64_t r) {
        const int slot = (int)(r % kCrtRecSlots);
        mbar_arrive_expect_tx(&full[slot], (uint32_t)S * cb);
        const uint8_t* src = R + row_of(r) * ldr + j0;
#pragma unroll
        for (int t = 0; t < S; ++t) bulk_load(slots[slot][t], src + (int64_t)t * rplane, cb, &full[slot]);
    };
    if (threadIdx.x == 0) {
        for (int i = 0; i < kCrtRecSlots; ++i) mbar_init(&full[i], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int64_t r = 0; r < nrows && r < kCrtRecSlots; ++r) issue(r);
    int fj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) fj[u] = jt + u < N ? __ldg(f + jt + u) : 0;
    const bool cfull = jt + 3 < N;
    int64_t r = 0;
    for (; r < nrows; ++r) {
        const int slot = (int)(r % kCrtRecSlots);
        bool ok = mbar_wait_bounded(&full[slot], (uint32_t)(r / kCrtRecSlots) & 1, tmo, nullptr, err);
        uint32_t v[S];
#pragma unroll
        for (int t = 0; t < S; ++t) v[t] = *reinterpret_cast<const uint32_t*>(&slots[slot][t][4 * threadIdx.x]);
        // all threads have read the slot (and agree that it had arrived)
        ok = __syncthreads_and(ok) != 0;
        if (!ok) break;
        if (threadIdx.x == 0 && r + kCrtRecSlots < nrows) {
            fence_proxy_async_smem();
            issue(r + kCrtRecSlots);
        }
        if (jt >= N) continue;
        const int64_t i = row_of(r);
        const int ei = e[i] - 2 * cc.k;
        double* ci = C + i * ldc + jt;
        int64_t hi[4];
        uint64_t lo[4];
        crt_reconstruct4<S>(v, cc, hi, lo);
        double o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            // a column past N computes from padding bytes and is not stored
            const double w = i128_scaled_to_double_rn(hi[u], lo[u], ei + fj[u]);
            o[u] = amode == 0 ? w : amode == 1 ? -w : alpha * w;
        }
        if (bmode) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (cfull || jt + u < N) o[u] = __fma_rn(beta, ci[u], o[u]);
        }
        if (cfull && (reinterpret_cast<uintptr_t>(ci) & 15) == 0) {
            reinterpret_cast<double2*>(ci)[0] = make_double2(o[0], o[1]);
            reinterpret_cast<double2*>(ci)[1] = make_double2(o[2], o[3]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (cfull || jt + u < N) ci[u] = o[u];
        }
    }
    if (r < nrows && threadIdx.x == 0) {
        // aborted: the copies already issued (rows r .. r + slots - 1) must
        // land before the block's shared memory goes away
        for (int64_t q = r; q < nrows && q < r + kCrtRecSlots; ++q)
            mbar_wait_bounded(&full[q % kCrtRecSlots], (uint32_t)(q / kCrtRecSlots) & 1, tmo,
                              nullptr, err, false);
    }
}

alp_status launch_recombine_crt(int n, int k, dim3 grid, cudaStream_t st, const uint8_t* R,
                                int64_t rplane, int64_t ldr, const int32_t* e, const int32_t* f,
                                int64_t M, int64_t N, double alpha, double beta, double* C,
                                int64_t ldc) {
    if (k < 1 || k > 60) return ALP_ERR_UNSUPPORTED;
    const CrtRecConsts cc = crt_rec_consts(n, k);
    const bool rvec = (reinterpret_cast<uintptr_t>(R) & 3) == 0 && rplane % 4 == 0 && ldr % 4 == 0;
    const bool staged =
        (reinterpret_cast<uintptr_t>(R) & 15) == 0 && rplane % 16 == 0 && ldr % 16 == 0;
    const int amode = alpha == 1.0 ? 0 : alpha == -1.0 ? 1 : 2;
    const int bmode = beta != 0.0 ? 1 : 0;
    const uint64_t tmo = wait_timeout_ns();
    int* err = device_error_word();
    // four columns per thread, 128-thread blocks: 512 columns per block, as
    // the grid was sized
#define ALP_CRT_REC_CASE(x)                                                                       \
    case x:                                                                                      \
        if (staged)                                                                              \
            recombine_crt_staged_kernel<x><<<grid, 128, 0, st>>>(                                 \
                R, rplane, ldr, e, f, M, N, alpha, beta, C, ldc, amode, bmode, cc, tmo, err);    \
        else                                                                                     \
            recombine_crt_kernel<x><<<grid, 128, 0, st>>>(R, rplane, ldr, e, f, M, N, alpha,     \
                                                          beta, C, ldc, rvec, amode, bmode, cc); \
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
