// Chinese remainder reconstruction of the modular emulated GEMM (the
// reconstruction kernel in emul_crt.cu).
//
// The tensor-core stage leaves, per element, the n bytes x_l = (P y_l) mod m_l
// with y_l = (Mn / m_l)^-1 mod m_l, so that sum_l x_l Mn / m_l = P + c Mn for
// an integer c.  The moduli are taken in groups of up to three, g = {l, l', l''}
// with product m_g <= 2^24: X_g = sum_{l in g} x_l m_g / m_l (< 3 m_g, 26 bits)
// gives sum_g X_g Mn / m_g = sum_l x_l Mn / m_l, so one 128-bit multiply-add
// with Mn / m_g (three or four 32-bit limbs) serves three moduli.  c is the
// nearest integer to sum_g X_g / m_g, formed in 6.58 fixed point from
// F_g = round(2^58 / m_g) with an error below 2^-30 (|P| / Mn <= 1/2 - 2^-19 by
// the choice of k, so the rounding is exact), and P = sum - c Mn follows by one
// carry pass, exact modulo 2^128, which holds it.
#pragma once

#include <cstdint>

#include "crt.cuh"
#include "emul_split.cuh"

namespace alp {

constexpr int kCrtMaxGroups = 6;   // ceil(16 / 3)

struct CrtRecConsts {
    uint32_t mn[4];                   // Mn, 32-bit limbs
    uint32_t mg[kCrtMaxGroups][4];    // Mn / m_g per group
    uint32_t fg_lo[kCrtMaxGroups];    // F_g = round(2^58 / m_g), low and high words
    uint32_t fg_hi[kCrtMaxGroups];
    uint32_t cl[16];                  // m_g / m_l for modulus l of group g
    int n, k;
};

// Host: the constants for n moduli and k bits (emul_crt.cu).
CrtRecConsts crt_rec_consts(int n, int k);

__device__ __forceinline__ uint64_t crt_mad_wide(uint32_t a, uint32_t b, uint64_t c) {
    uint64_t d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// P (signed 128-bit hi:lo) of four adjacent columns whose residue bytes are
// the bytes of v[l], l < S (byte u = column u).  Every group's constants are
// read once for the four columns.  The limbs of Mn / m_g that can be nonzero:
// Mn / m_g < 2^24, 2^48, 2^72, 2^95 for S <= 6, 9, 12, 15 (one to three
// limbs), 2^118 for S = 16 (four).
template <int S>
__device__ __forceinline__ void crt_reconstruct4(const uint32_t (&v)[S], const CrtRecConsts& cc,
                                                 int64_t (&hi)[4], uint64_t (&lo)[4]) {
    constexpr int G = (S + 2) / 3;
    constexpr int kLimbs = S <= 6 ? 1 : S <= 9 ? 2 : S <= 15 ? 3 : 4;
    uint64_t a0[4], a1[4], a2[4], a3[4], q[4];
    uint32_t qh[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a0[u] = a1[u] = a2[u] = a3[u] = q[u] = 0, qh[u] = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        // X_g by two-way dot products: every weight m_g / m_l is a product of
        // at most two moduli <= 256 * 255 < 2^16, so the first two moduli of
        // the group share one 16-bit weight pair and one permuted word of
        // residue bytes per two columns (bytes x_a, x_b of column u at 2u,
        // 2u + 1 of the pair word); the third adds its bytes with a zero
        // partner.
        const int a = 3 * g, b = a + 1, c = a + 2;
        const uint32_t wab = cc.cl[a] | (b < S ? cc.cl[b] << 16 : 0u);
        const uint32_t vb = b < S ? v[b < S ? b : a] : 0u;
        const uint32_t p01 = __byte_perm(v[a], vb, 0x5140u);
        const uint32_t p23 = __byte_perm(v[a], vb, 0x7362u);
        uint32_t X[4] = {__dp2a_lo(wab, p01, 0u), __dp2a_hi(wab, p01, 0u),
                         __dp2a_lo(wab, p23, 0u), __dp2a_hi(wab, p23, 0u)};
        if (c < S) {
            const uint32_t wc = cc.cl[c < S ? c : a];
            const uint32_t vc = v[c < S ? c : a];
            const uint32_t q01 = __byte_perm(vc, 0u, 0x4140u);
            const uint32_t q23 = __byte_perm(vc, 0u, 0x4342u);
            X[0] = __dp2a_lo(wc, q01, X[0]);
            X[1] = __dp2a_hi(wc, q01, X[1]);
            X[2] = __dp2a_lo(wc, q23, X[2]);
            X[3] = __dp2a_hi(wc, q23, X[3]);
        }
        const uint32_t m0 = cc.mg[g][0], m1 = cc.mg[g][1], m2 = cc.mg[g][2], m3 = cc.mg[g][3];
        const uint32_t f0 = cc.fg_lo[g], f1 = cc.fg_hi[g];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a0[u] = crt_mad_wide(X[u], m0, a0[u]);
            if (kLimbs > 1) a1[u] = crt_mad_wide(X[u], m1, a1[u]);
            if (kLimbs > 2) a2[u] = crt_mad_wide(X[u], m2, a2[u]);
            if (kLimbs > 3) a3[u] = crt_mad_wide(X[u], m3, a3[u]);
            q[u] = crt_mad_wide(X[u], f0, q[u]);
            qh[u] += X[u] * f1;
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        // sum_g X_g F_g < 2^62 (X_g / m_g < 3, at most six groups), so its
        // value modulo 2^64 is the value
        const uint64_t qt = q[u] + ((uint64_t)qh[u] << 32);
        const uint32_t c = (uint32_t)((qt + (1ull << 57)) >> 58);
        // the column sums are below 6 * 2^26 * 2^32 < 2^61: signed 64-bit
        // holds each step of the carry pass
        int64_t t = (int64_t)a0[u] - (int64_t)((uint64_t)c * cc.mn[0]);
        const uint32_t w0 = (uint32_t)t;
        t = (t >> 32) + (int64_t)a1[u] - (int64_t)((uint64_t)c * cc.mn[1]);
        const uint32_t w1 = (uint32_t)t;
        t = (t >> 32) + (int64_t)a2[u] - (int64_t)((uint64_t)c * cc.mn[2]);
        const uint32_t w2 = (uint32_t)t;
        t = (t >> 32) + (int64_t)a3[u] - (int64_t)((uint64_t)c * cc.mn[3]);
        const uint32_t w3 = (uint32_t)t;
        hi[u] = (int64_t)(((uint64_t)w3 << 32) | w2);
        lo[u] = ((uint64_t)w1 << 32) | w0;
    }
}

// The same for a modulus count n (4..16) known only at run time: v[l] = 0
// and the constants of moduli l >= n are zero (crt_rec_consts zero-fills
// them), so a group or limb past the count adds nothing; groups wholly past
// it are skipped (n is the same in every thread), and the fourth limb is
// formed for n = 16 only.  Used where one kernel serves every count.
__device__ __forceinline__ void crt_reconstruct4_n(const uint32_t (&v)[16], int n,
                                                   const CrtRecConsts& cc, int64_t (&hi)[4],
                                                   uint64_t (&lo)[4]) {
    uint64_t a0[4], a1[4], a2[4], a3[4], q[4];
    uint32_t qh[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a0[u] = a1[u] = a2[u] = a3[u] = q[u] = 0, qh[u] = 0;
    const bool four = n > 15;
#pragma unroll
    for (int g = 0; g < kCrtMaxGroups; ++g) {
        if (3 * g >= n) break;
        const int a = 3 * g, b = a + 1, c = a + 2;
        const uint32_t wab = cc.cl[a] | (b < 16 ? cc.cl[b < 16 ? b : a] << 16 : 0u);
        const uint32_t vb = b < 16 ? v[b < 16 ? b : a] : 0u;
        const uint32_t p01 = __byte_perm(v[a], vb, 0x5140u);
        const uint32_t p23 = __byte_perm(v[a], vb, 0x7362u);
        uint32_t X[4] = {__dp2a_lo(wab, p01, 0u), __dp2a_hi(wab, p01, 0u),
                         __dp2a_lo(wab, p23, 0u), __dp2a_hi(wab, p23, 0u)};
        if (c < 16) {
            const uint32_t wc = cc.cl[c < 16 ? c : a];
            const uint32_t vc = v[c < 16 ? c : a];
            const uint32_t q01 = __byte_perm(vc, 0u, 0x4140u);
            const uint32_t q23 = __byte_perm(vc, 0u, 0x4342u);
            X[0] = __dp2a_lo(wc, q01, X[0]);
            X[1] = __dp2a_hi(wc, q01, X[1]);
            X[2] = __dp2a_lo(wc, q23, X[2]);
            X[3] = __dp2a_hi(wc, q23, X[3]);
        }
        const uint32_t m0 = cc.mg[g][0], m1 = cc.mg[g][1], m2 = cc.mg[g][2], m3 = cc.mg[g][3];
        const uint32_t f0 = cc.fg_lo[g], f1 = cc.fg_hi[g];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a0[u] = crt_mad_wide(X[u], m0, a0[u]);
            a1[u] = crt_mad_wide(X[u], m1, a1[u]);
            a2[u] = crt_mad_wide(X[u], m2, a2[u]);
            if (four) a3[u] = crt_mad_wide(X[u], m3, a3[u]);
            q[u] = crt_mad_wide(X[u], f0, q[u]);
            qh[u] += X[u] * f1;
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        // as in crt_reconstruct4
        const uint64_t qt = q[u] + ((uint64_t)qh[u] << 32);
        const uint32_t c = (uint32_t)((qt + (1ull << 57)) >> 58);
        int64_t t = (int64_t)a0[u] - (int64_t)((uint64_t)c * cc.mn[0]);
        const uint32_t w0 = (uint32_t)t;
        t = (t >> 32) + (int64_t)a1[u] - (int64_t)((uint64_t)c * cc.mn[1]);
        const uint32_t w1 = (uint32_t)t;
        t = (t >> 32) + (int64_t)a2[u] - (int64_t)((uint64_t)c * cc.mn[2]);
        const uint32_t w2 = (uint32_t)t;
        t = (t >> 32) + (int64_t)a3[u] - (int64_t)((uint64_t)c * cc.mn[3]);
        const uint32_t w3 = (uint32_t)t;
        hi[u] = (int64_t)(((uint64_t)w3 << 32) | w2);
        lo[u] = ((uint64_t)w1 << 32) | w0;
    }
}

}  // namespace alp
