// The moduli of the modular emulated GEMM and reduction modulo them, shared by
// the split, the tensor-core epilogue and the reconstruction.
#pragma once

#include <cstdint>

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
// ceil(2^38 / m): x mod m = x - floor(x magic / 2^38) m for x < 2^30.  The
// product over-estimates x / m by less than x / 2^38 < 2^-8 <= 1/m, and the
// fraction of x / m is at most 1 - 1/m, so the floor is exact; for m = 256
// the magic is 2^30 and the quotient is x >> 8.
__host__ __device__ __forceinline__ constexpr uint32_t crt_magic(uint32_t m) {
    return (uint32_t)(((1ull << 38) + m - 1) / m);
}
// x mod m for x < 2^30.
__device__ __forceinline__ uint32_t crt_mod(uint32_t x, uint32_t m, uint32_t magic) {
    return x - (__umulhi(x, magic) >> 6) * m;
}
__device__ __forceinline__ uint32_t crt_mod(uint32_t x, uint32_t m) {
    return crt_mod(x, m, crt_magic(m));
}
// Q mod m in [0, m) for a signed |Q| < 2^30.
__device__ __forceinline__ uint32_t crt_residue(int32_t Q, uint32_t m, uint32_t magic) {
    const uint32_t a = Q < 0 ? 0u - (uint32_t)Q : (uint32_t)Q;
    const uint32_t r = crt_mod(a, m, magic);
    return (Q < 0 && r) ? m - r : r;
}

}  // namespace alp
