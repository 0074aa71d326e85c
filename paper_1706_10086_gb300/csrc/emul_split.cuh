// Device helpers of the emulated GEMMs: the exact fixed-point form of a
// scaled operand, its digits, bf16 packing, the split kernels (rows of a
// row-major matrix, or its columns through shared memory), which take a
// splitter object that turns one value into S small integers and packs two
// of them into bf16, and the rounding of a 128-bit integer to double.
#pragma once

#include <cuda_bf16.h>

#include "alp_internal.cuh"

namespace alp {

// The frexp exponent of a double given by its bits without the sign: the e
// with 2^(e-1) <= |x| < 2^e (0 for zero).
__device__ __forceinline__ int frexp_exponent_of_bits(uint64_t mb) {
    if (mb == 0) return 0;
    const int ex = (int)(mb >> 52);
    if (ex == 0) return (63 - __clzll((long long)mb)) - 1073;   // subnormal
    return ex - 1022;
}

// ---------------------------------------------------------------------------
// 2. split
// ---------------------------------------------------------------------------
// Digits of a * 2^-e.  r0 = a * 2^-e is held as a 64-bit fixed-point number
// with 62 fraction bits, rounded to odd (truncate, then set the last bit if
// anything was cut off): every later rounding happens at least 2 bits above
// that last bit, so the digits equal those of the exact value ((s-1) b + 2 <=
// 62 - b).  Each step is d = round-half-even(X / 2^(62-b)), X = (X - d 2^(62-b))
// * 2^b, which is x = r * 2^b, d = nearest integer (ties to even), r = x - d in
// fixed point.
__device__ __forceinline__ uint64_t fixed_point_r0(double a, int e) {
    const uint64_t bits = (uint64_t)__double_as_longlong(a);
    const bool neg = (bits >> 63) != 0;
    const int ex = (int)((bits >> 52) & 0x7FF);
    uint64_t m = bits & ((1ull << 52) - 1);
    int E;
    if (ex == 0x7FF) {
        m = 0;
        E = 0;   // Inf/NaN: reported by the scan; digits 0
    } else if (ex == 0) {
        E = -1074;
    } else {
        m |= 1ull << 52;
        E = ex - 1075;
    }
    const int sh = E - e + 62;
    uint64_t Y;
    if (m == 0) Y = 0;
    else if (sh >= 0) Y = m << (sh > 63 ? 63 : sh);
    else if (sh > -64) {
        const int r = -sh;
        Y = (m >> r) | ((m & ((1ull << r) - 1)) != 0 ? 1ull : 0ull);
    } else Y = 1;   // nonzero but below 2^-62: sticky bit only
    return neg ? (0ull - Y) : Y;   // two's complement of the signed value
}

template <int S, int B>
__device__ __forceinline__ void split_digits(double a, int e, int (&d)[S]) {
    constexpr int SH = 62 - B;   // the digit's unit in the fixed point
    uint64_t X = fixed_point_r0(a, e);
#pragma unroll
    for (int p = 0; p < S; ++p) {
        // round half to even of X / 2^SH: floor((X + 2^(SH-1) - 1 + odd) / 2^SH),
        // odd = the parity of floor(X / 2^SH)
        const uint64_t odd = (X >> SH) & 1;
        const int64_t dd = (int64_t)(X + ((1ull << (SH - 1)) - 1) + odd) >> SH;
        d[p] = (int)dd;
        // (X - dd 2^SH) 2^B, |.| <= 2^61; SH + B = 62
        X = (X << B) - ((uint64_t)dd << 62);
    }
}

// The splitter of the digit schemes: s digits of B bits (split_digits).  The
// split kernels below take a splitter object, so that other integer
// representations of the operands (the residues of the modular scheme) reuse
// them.
// Two digits (|v| <= 256) as packed bf16: the float 1.5*2^23 + v - 1.5*2^23
// is exactly v, and its upper 16 bits are its bf16 encoding (at most 9
// significant bits), so no conversion instruction is needed.
__device__ __forceinline__ uint32_t pack_bf16x2(int lo, int hi) {
    const float fl = __int_as_float(0x4B400000 + lo) - 12582912.0f;
    const float fh = __int_as_float(0x4B400000 + hi) - 12582912.0f;
    return __byte_perm((uint32_t)__float_as_int(fl), (uint32_t)__float_as_int(fh), 0x7632);
}

template <int B>
struct DigitSplit {
    template <int S>
    __device__ __forceinline__ void split(double a, int e, int (&d)[S]) const {
        split_digits<S, B>(a, e, d);
    }
    __device__ __forceinline__ uint32_t pack(int lo, int hi) const { return pack_bf16x2(lo, hi); }
};

// A (R x K, row-major) -> out[p][r][k] (row stride kpad, zero beyond K); each
// thread handles two consecutive k.
template <typename T, int S, typename Sp>
__global__ void split_rows_kernel(const T* __restrict__ X, int64_t R, int64_t K,
                                  int64_t ldx, const int32_t* __restrict__ e,
                                  __nv_bfloat16* __restrict__ out, int64_t kpad, const Sp sp) {
    const int64_t half = kpad >> 1;
    const int64_t total = R * half;
    const int64_t plane = R * kpad;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / half;
        const int64_t k = (idx - r * half) * 2;
        const int er = e[r];
        int d0[S], d1[S];
        sp.template split<S>(k < K ? (double)__ldg(X + r * ldx + k) : 0.0, er, d0);
        sp.template split<S>(k + 1 < K ? (double)__ldg(X + r * ldx + k + 1) : 0.0, er, d1);
        uint32_t* o = reinterpret_cast<uint32_t*>(out + r * kpad + k);
#pragma unroll
        for (int p = 0; p < S; ++p, o += plane >> 1) *o = sp.pack(d0[p], d1[p]);
    }
}

// As split_rows_kernel with four consecutive k per thread: rows from
// blockIdx.y (grid stride, no division per element), two 16-byte loads of A
// when its row is 16-byte aligned, one 8-byte store per digit plane.  Needs
// out 8-byte aligned (the launch checks).  THREADS and MINB are the launch's
// block size and the blocks per SM its register budget must allow.
template <typename T, int S, typename Sp, int THREADS = 256, int MINB = 1>
__global__ void __launch_bounds__(THREADS, MINB) split_rows4_kernel(const T* __restrict__ X, int64_t R,
                                                          int64_t K, int64_t ldx,
                                                          const int32_t* __restrict__ e,
                                                          __nv_bfloat16* __restrict__ out,
                                                          int64_t kpad, const Sp sp) {
    const int64_t plane = R * kpad;
    for (int64_t r = blockIdx.y; r < R; r += gridDim.y) {
        const int er = e[r];
        const T* xr = X + r * ldx;
        const bool xvec = (reinterpret_cast<uintptr_t>(xr) & 15) == 0;
        for (int64_t k = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); k < kpad;
             k += 4 * (int64_t)gridDim.x * blockDim.x) {
            double a[4];
            if (xvec && k + 3 < K) {
                if constexpr (sizeof(T) == 8) {
                    const double2 p0 = __ldg(reinterpret_cast<const double2*>(xr + k));
                    const double2 p1 = __ldg(reinterpret_cast<const double2*>(xr + k + 2));
                    a[0] = p0.x;
                    a[1] = p0.y;
                    a[2] = p1.x;
                    a[3] = p1.y;
                } else {
                    const float4 p0 = __ldg(reinterpret_cast<const float4*>(xr + k));
                    a[0] = p0.x;
                    a[1] = p0.y;
                    a[2] = p0.z;
                    a[3] = p0.w;
                }
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = k + u < K ? (double)__ldg(xr + k + u) : 0.0;
            }
            // pairs packed as soon as they are split, so that only the packed
            // words of the first pair stay live
            uint32_t w01[S];
            {
                int d0[S], d1[S];
                sp.template split<S>(a[0], er, d0);
                sp.template split<S>(a[1], er, d1);
#pragma unroll
                for (int p = 0; p < S; ++p) w01[p] = sp.pack(d0[p], d1[p]);
            }
            int d2[S], d3[S];
            sp.template split<S>(a[2], er, d2);
            sp.template split<S>(a[3], er, d3);
            uint2* o = reinterpret_cast<uint2*>(out + r * kpad + k);
#pragma unroll
            for (int p = 0; p < S; ++p, o += plane >> 2) *o = make_uint2(w01[p], sp.pack(d2[p], d3[p]));
        }
    }
}

// The row exponent scan and split_rows4_kernel in one kernel, one block per
// row at a time (double operands): pass 1 reads the row in the split's own
// pattern for the largest magnitude (the block's maximum through one shared
// slot per row parity, one barrier per row), which gives e_r (stored, and an
// Inf/NaN recorded in the error word as the scan does); pass 2 splits the row
// with it, its loads served by L2.  Needs out 8-byte aligned and kpad a
// multiple of 4 (the launch checks).
template <int S, typename Sp, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) scan_split_rows4_kernel(
    const double* __restrict__ X, int64_t R, int64_t K, int64_t ldx, int32_t* __restrict__ e,
    __nv_bfloat16* __restrict__ out, int64_t kpad, const Sp sp, int* err) {
    __shared__ uint64_t red[2][THREADS / 32];
    const int64_t plane = R * kpad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int par = 0;
    for (int64_t r = blockIdx.x; r < R; r += gridDim.x, par ^= 1) {
        const double* xr = X + r * ldx;
        const bool xvec = (reinterpret_cast<uintptr_t>(xr) & 15) == 0;
        uint64_t mx = 0;
        // four strides of the row per iteration, all their loads issued
        // before the first comparison (the scan is bound by load latency)
#pragma unroll 1
        for (int64_t k0 = 4 * (int64_t)threadIdx.x; k0 < K; k0 += 16 * THREADS) {
            uint64_t b[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t k = k0 + (int64_t)q * 4 * THREADS;
                if (xvec && k + 3 < K) {
                    const uint4 p0 = __ldg(reinterpret_cast<const uint4*>(xr + k));
                    const uint4 p1 = __ldg(reinterpret_cast<const uint4*>(xr + k + 2));
                    b[4 * q] = ((uint64_t)p0.y << 32) | p0.x;
                    b[4 * q + 1] = ((uint64_t)p0.w << 32) | p0.z;
                    b[4 * q + 2] = ((uint64_t)p1.y << 32) | p1.x;
                    b[4 * q + 3] = ((uint64_t)p1.w << 32) | p1.z;
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        b[4 * q + u] =
                            k + u < K ? (uint64_t)__double_as_longlong(__ldg(xr + k + u)) : 0ull;
                }
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const uint64_t a = b[u] & 0x7FFFFFFFFFFFFFFFull;
                mx = a > mx ? a : mx;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t y = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = y > mx ? y : mx;
        }
        if (lane == 0) red[par][warp] = mx;
        __syncthreads();
        mx = red[par][0];
#pragma unroll
        for (int w = 1; w < THREADS / 32; ++w) mx = red[par][w] > mx ? red[par][w] : mx;
        const int er = frexp_exponent_of_bits(mx);
        if (threadIdx.x == 0) {
            e[r] = er;
            if (mx >= 0x7FF0000000000000ull) set_device_error(err, ALP_ERR_UNSUPPORTED);
        }
        // the split: the next stride's four values loaded before this
        // stride's residues are formed (the row comes back from L2)
        auto load4 = [&](int64_t k, double (&a)[4]) {
            if (xvec && k + 3 < K) {
                const double2 p0 = __ldg(reinterpret_cast<const double2*>(xr + k));
                const double2 p1 = __ldg(reinterpret_cast<const double2*>(xr + k + 2));
                a[0] = p0.x;
                a[1] = p0.y;
                a[2] = p1.x;
                a[3] = p1.y;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = k + u < K ? __ldg(xr + k + u) : 0.0;
            }
        };
        double an[4];
        if (4 * (int64_t)threadIdx.x < kpad) load4(4 * (int64_t)threadIdx.x, an);
#pragma unroll 1
        for (int64_t k = 4 * (int64_t)threadIdx.x; k < kpad; k += 4 * THREADS) {
            const double a[4] = {an[0], an[1], an[2], an[3]};
            if (k + 4 * THREADS < kpad) load4(k + 4 * THREADS, an);
            uint32_t w01[S];
            {
                int d0[S], d1[S];
                sp.template split<S>(a[0], er, d0);
                sp.template split<S>(a[1], er, d1);
#pragma unroll
                for (int p = 0; p < S; ++p) w01[p] = sp.pack(d0[p], d1[p]);
            }
            int d2[S], d3[S];
            sp.template split<S>(a[2], er, d2);
            sp.template split<S>(a[3], er, d3);
            uint2* o = reinterpret_cast<uint2*>(out + r * kpad + k);
#pragma unroll
            for (int p = 0; p < S; ++p, o += plane >> 2) *o = make_uint2(w01[p], sp.pack(d2[p], d3[p]));
        }
    }
}

// B (K x N, row-major) -> out[p][j][k] (row stride kpad): 64 x 32 tiles through
// shared memory so that reads run along j and writes along k.
template <typename T, int S, typename Sp>
__global__ void split_cols_kernel(const T* __restrict__ X, int64_t K, int64_t N,
                                  int64_t ldx, const int32_t* __restrict__ f,
                                  __nv_bfloat16* __restrict__ out, int64_t kpad, const Sp sp) {
    __shared__ double t[32][65];
    const int64_t j0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 64;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 warps
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t k = k0 + ty + 8 * r, j = j0 + tx;
        t[tx][ty + 8 * r] = (k < K && j < N) ? (double)__ldg(X + k * ldx + j) : 0.0;
    }
    __syncthreads();
    const int64_t plane = N * kpad;
#pragma unroll
    for (int jj = ty; jj < 32; jj += 8) {
        const int64_t j = j0 + jj;
        if (j >= N) continue;
        const int fj = f[j];
        int d0[S], d1[S];
        sp.template split<S>(t[jj][2 * tx], fj, d0);
        sp.template split<S>(t[jj][2 * tx + 1], fj, d1);
        const int64_t k = k0 + 2 * tx;
        if (k >= kpad) continue;
        uint32_t* o = reinterpret_cast<uint32_t*>(out + j * kpad + k);
#pragma unroll
        for (int p = 0; p < S; ++p, o += plane >> 1) *o = sp.pack(d0[p], d1[p]);
    }
}

// As split_cols_kernel with four consecutive k per thread: 128 x 32 tiles, the
// tile row of column jj holding k = 4q + i at position 32 i + q (q < 32, i <
// 4), so that the tile's fill (one k of 32 columns per warp, a row stride of
// 129 doubles) and the reads of four consecutive k by each lane (32
// consecutive doubles per access) are free of bank conflicts; one 8-byte store
// per digit plane (256 contiguous bytes per warp).  Needs out 8-byte aligned
// and kpad a multiple of 4 (the launch checks).
template <typename T, int S, typename Sp>
__global__ void __launch_bounds__(256, 3) split_cols4_kernel(
    const T* __restrict__ X, int64_t K, int64_t N, int64_t ldx, const int32_t* __restrict__ f,
    __nv_bfloat16* __restrict__ out, int64_t kpad, const Sp sp) {
    __shared__ double t[32][129];
    const int64_t j0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 128;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 warps
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int kk = ty + 8 * r;
        const int64_t k = k0 + kk, j = j0 + tx;
        t[tx][(kk & 3) * 32 + (kk >> 2)] = (k < K && j < N) ? (double)__ldg(X + k * ldx + j) : 0.0;
    }
    __syncthreads();
    const int64_t plane = N * kpad;
    const int64_t k = k0 + 4 * tx;
    if (k >= kpad) return;
#pragma unroll 1
    for (int jj = ty; jj < 32; jj += 8) {
        const int64_t j = j0 + jj;
        if (j >= N) break;
        const int fj = f[j];
        uint32_t w01[S];
        {
            int d0[S], d1[S];
            sp.template split<S>(t[jj][tx], fj, d0);
            sp.template split<S>(t[jj][32 + tx], fj, d1);
#pragma unroll
            for (int p = 0; p < S; ++p) w01[p] = sp.pack(d0[p], d1[p]);
        }
        int d2[S], d3[S];
        sp.template split<S>(t[jj][64 + tx], fj, d2);
        sp.template split<S>(t[jj][96 + tx], fj, d3);
        uint2* o = reinterpret_cast<uint2*>(out + j * kpad + k);
#pragma unroll
        for (int p = 0; p < S; ++p, o += plane >> 2) *o = make_uint2(w01[p], sp.pack(d2[p], d3[p]));
    }
}

// Nearest double (ties to even) of the 128-bit two's-complement integer
// hi:lo, multiplied by 2^E: built from 64-bit integer operations on the IEEE
// encoding (FP64 arithmetic is slow on this GPU), with selects instead of
// branches for the sign and the rounding (they differ between neighbouring
// elements).  When the scaled result would leave the normal range it falls
// back to ldexp of the rounded value (which rounds a subnormal result a second
// time, as the definition does).
__device__ __forceinline__ double i128_scaled_to_double_rn(int64_t hi_s, uint64_t lo, int E) {
    // magnitude: (x XOR s) - s with s = 0 or all ones, a 128-bit subtraction
    const uint64_t sgn = (uint64_t)(hi_s >> 63);
    uint64_t l = lo ^ sgn, h = (uint64_t)hi_s ^ sgn;
    asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %2;" : "+l"(l), "+l"(h) : "l"(sgn));
    const bool zero = (h | l) == 0;   // selected at the end, not branched on
    // top: the 64 bits from the leading one down; sticky: any one bit below
    const bool hz = h == 0;
    const uint64_t x = hz ? l : h, y = hz ? 0ull : l;
    const int nz = __clzll((long long)x) & 63;   // 64 only for zero
    const uint64_t top = (x << nz) | ((y >> 1) >> (63 - nz));
    const uint32_t sticky = (y << nz) != 0 ? 1u : 0u;
    int msb = (hz ? 63 : 127) - nz;
    uint64_t m = top >> 11;                      // 53 bits, leading one at bit 52
    const uint32_t low = (uint32_t)top & 0x7FFu;
    const uint32_t up = (low > 0x400u ? 1u : 0u) |
                        (low == 0x400u ? (sticky | ((uint32_t)m & 1u)) : 0u);
    m += up;
    const uint32_t carry = (uint32_t)(m >> 53);  // rounded up to 2^53
    m >>= carry;
    msb += (int)carry;
    // m in [2^52, 2^53): value = m * 2^(msb - 52) * 2^E
    const int be = msb + E + 1023;
    const uint64_t frac = m & ((1ull << 52) - 1);
    if (zero) return 0.0;
    if (be >= 1 && be <= 2046)
        return __longlong_as_double((long long)((sgn << 63) | ((uint64_t)be << 52) | frac));
    const double v = __longlong_as_double(
        (long long)((sgn << 63) | ((uint64_t)(msb + 1023) << 52) | frac));
    return ldexp(v, E);
}

}  // namespace alp
