// Device building blocks of the native FP64 GEMM, shared by the single-GEMM
// kernels (native.cu) and the batched persistent kernel (batched.cu).
#pragma once

#include "alp_internal.cuh"
#include "native_cfg.h"

namespace alp {

// Per-thread accumulator tile: (tm/2) x (tn/2) DMMA fragments of 4 doubles.
template <int TM, int TN>
struct Acc {
    double c[TM / 2][TN / 2][4];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < TM / 2; ++i)
#pragma unroll
            for (int j = 0; j < TN / 2; ++j)
#pragma unroll
                for (int r = 0; r < 4; ++r) c[i][j][r] = 0.0;
    }
};

// One shared-memory stage of the tile product (the inner loop of Fig. 2):
// As is a bm x bk tile (row-major, row length bk), Bs a bk x bn tile (row
// length bn).  The warp's tile starts at row wm0 of As and column wn0 of Bs.
template <int TM, int TN>
__device__ __forceinline__ void mma_stage(const double* __restrict__ As,
                                          const double* __restrict__ Bs, int bk, int bn,
                                          int wm0, int wn0, int lane, Acc<TM, TN>& acc) {
    const int g = lane >> 2, t = lane & 3;
    const double* a_base = As + (wm0 + g) * bk + t;
    const double* b_base = Bs + t * bn + wn0 + g;
#pragma unroll 2
    for (int kk = 0; kk < bk; kk += 4) {
        double a[TM / 2][2], b[TN / 2];
#pragma unroll
        for (int mi = 0; mi < TM / 2; ++mi) {
            a[mi][0] = a_base[(mi * 16) * bk + kk];
            a[mi][1] = a_base[(mi * 16 + 8) * bk + kk];
        }
#pragma unroll
        for (int ni = 0; ni < TN / 2; ++ni) b[ni] = b_base[kk * bn + ni * 8];
#pragma unroll
        for (int mi = 0; mi < TM / 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < TN / 2; ++ni) dmma_16x8x4(acc.c[mi][ni], a[mi][0], a[mi][1], b[ni]);
    }
}

// Epilogue (Fig. 2 caption: C is read and written once): C = alpha*acc + beta*C
// for the thread's fragments, rows/columns outside M x N skipped.  beta == 0
// reads no C.  vec2: C and ldc allow 16-byte accesses at even columns.
template <int TM, int TN>
__device__ __forceinline__ void epilogue(const Acc<TM, TN>& acc, double* __restrict__ C,
                                         int64_t ldc, int64_t M, int64_t N, int64_t row0,
                                         int64_t col0, double alpha, double beta, bool vec2,
                                         int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < TM / 2; ++mi) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t r = row0 + mi * 16 + g + h * 8;
            if (r >= M) continue;
            double* crow = C + r * ldc;
#pragma unroll
            for (int ni = 0; ni < TN / 2; ++ni) {
                const int64_t c = col0 + ni * 8 + 2 * t;
                double v0 = alpha * acc.c[mi][ni][2 * h + 0];
                double v1 = alpha * acc.c[mi][ni][2 * h + 1];
                if (vec2 && c + 1 < N) {
                    double2* p = reinterpret_cast<double2*>(crow + c);
                    if (beta != 0.0) {
                        double2 old = *p;
                        v0 = __fma_rn(beta, old.x, v0);
                        v1 = __fma_rn(beta, old.y, v1);
                    }
                    *p = make_double2(v0, v1);
                } else {
                    if (c < N) crow[c] = (beta != 0.0) ? __fma_rn(beta, crow[c], v0) : v0;
                    if (c + 1 < N) crow[c + 1] = (beta != 0.0) ? __fma_rn(beta, crow[c + 1], v1) : v1;
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------
// cp.async tile mainloop (no TMA): used where TMA's alignment rules do not hold
// and by the batched kernel, whose problems each have their own pointers.
// All threads of the block load; `S` stages; 8-byte copies with zero fill.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct TileProblem {
    const double* A;
    const double* B;
    double* C;
    int64_t lda, ldb, ldc, M, N, K;
    double alpha, beta;
};

__device__ __forceinline__ void load_tile_async(double* As, double* Bs, const TileProblem& p,
                                                int64_t m0, int64_t n0, int64_t k0, int bm,
                                                int bn, int bk, int tid, int nthreads) {
    for (int e = tid; e < bm * bk; e += nthreads) {
        const int r = e / bk, c = e - r * bk;
        const int64_t gr = m0 + r, gc = k0 + c;
        const bool ok = gr < p.M && gc < p.K;
        cp_async8(As + e, ok ? (p.A + gr * p.lda + gc) : p.A, ok);
    }
    for (int e = tid; e < bk * bn; e += nthreads) {
        const int r = e / bn, c = e - r * bn;
        const int64_t gr = k0 + r, gc = n0 + c;
        const bool ok = gr < p.K && gc < p.N;
        cp_async8(Bs + e, ok ? (p.B + gr * p.ldb + gc) : p.B, ok);
    }
}

// Computes one bm x bn tile of problem p at (m0, n0) with a 2-stage cp.async
// ring in `smem` (2 * (bm + bn) * bk doubles) and writes it out.  All threads
// of the block call it; warps beyond the tile's warp grid only help to load.
template <int TM, int TN>
__device__ __forceinline__ void tile_ldg(const TileProblem& p, int64_t m0, int64_t n0, int bm,
                                         int bn, int bk, double* smem, bool vec2) {
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int wn_count = bn / (4 * TN);
    const int nwarps_c = (bm / (8 * TM)) * wn_count;
    const int wm0 = (warp / wn_count) * 8 * TM, wn0 = (warp % wn_count) * 4 * TN;
    double* As[2] = {smem, smem + (bm + bn) * bk};
    double* Bs[2] = {smem + bm * bk, smem + (bm + bn) * bk + bm * bk};
    Acc<TM, TN> acc;
    acc.zero();
    const int64_t KT = (p.K + bk - 1) / bk;
    if (KT > 0) load_tile_async(As[0], Bs[0], p, m0, n0, 0, bm, bn, bk, tid, nthreads);
    cp_async_commit();
    for (int64_t kt = 0; kt < KT; ++kt) {
        const int s = (int)(kt & 1);
        if (kt + 1 < KT)
            load_tile_async(As[s ^ 1], Bs[s ^ 1], p, m0, n0, (kt + 1) * bk, bm, bn, bk, tid, nthreads);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        if (warp < nwarps_c) mma_stage<TM, TN>(As[s], Bs[s], bk, bn, wm0, wn0, lane, acc);
        __syncthreads();
    }
    cp_async_wait<0>();
    if (warp < nwarps_c)
        epilogue<TM, TN>(acc, p.C, p.ldc, p.M, p.N, m0 + wm0, n0 + wn0, p.alpha, p.beta, vec2, lane);
}

}  // namespace alp
