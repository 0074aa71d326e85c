// Native FP64 GEMM, C = alpha*A*B + beta*C (Eq. 1 of Matthes et al. 2017), on
// FP64 DMMA tensor-core MMAs.
//
// Kernel structure (the tiled algorithm of Sect. 2.1 / Fig. 2 re-designed for
// sm_103a): one thread block per bm x bn tile of C; warp 0 is a producer that
// streams bm x bk tiles of A and bk x bn tiles of B into an S-stage shared
// memory ring with TMA (cp.async.bulk.tensor, completion on "full" mbarriers);
// the remaining warps wait on "full", run the tile product with m16n8k4 DMMA
// into per-thread tm x tn register tiles, and release the stage on its "empty"
// mbarrier.  The epilogue streams alpha*acc + beta*C once.
//
// Every wait is bounded (ALP_ERR_TIMEOUT into the device error word); on abort
// the producer waits for the copies it issued before the block exits.

#include "native.cuh"

namespace alp {

struct NativeParams {
    int64_t M, N, K;
    double alpha, beta;
    double* C;
    int64_t ldc;
    int bm, bn, bk, stages;
    int tiles_m, tiles_n;
    int vec2;
    uint64_t timeout_ns;
    int* err;
    int inject_skip_kt;   // test hook: producer of block 0 skips this k-tile's copies (-1: off)
};

constexpr int kGroupM = 8;   // tile raster: 8 tile-rows per group, for L2 reuse of B panels

__device__ __forceinline__ void tile_coords(int pid, int tiles_m, int tiles_n, int& tm, int& tn) {
    const int in_group = kGroupM * tiles_n;
    const int group = pid / in_group;
    const int first_m = group * kGroupM;
    const int gsz = min(tiles_m - first_m, kGroupM);
    const int local = pid % in_group;
    tm = first_m + local % gsz;
    tn = local / gsz;
}

template <int TM, int TN>
__global__ void __launch_bounds__(max_threads(TM, TN), 1)
    dgemm_tma_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB, NativeParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int bm = p.bm, bn = p.bn, bk = p.bk, S = p.stages;
    double* tiles = reinterpret_cast<double*>(smem_raw);
    const int stage_elems = (bm + bn) * bk;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)stage_elems * 8 * S);
    uint64_t* empty = full + S;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_cwarps = (blockDim.x >> 5) - 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], n_cwarps);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();

    int tmi, tni;
    tile_coords(blockIdx.x, p.tiles_m, p.tiles_n, tmi, tni);
    const int64_t m0 = (int64_t)tmi * bm, n0 = (int64_t)tni * bn;
    const int64_t KT = (p.K + bk - 1) / bk;
    const uint32_t stage_bytes = (uint32_t)stage_elems * 8;

    if (warp == 0) {
        // ---------------- producer ----------------
        if (lane == 0) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
            int64_t issued = 0;           // k-tiles whose copies were issued
            int64_t skipped = -1;
            for (int64_t kt = 0; kt < KT; ++kt) {
                const int s = (int)(kt % S);
                const uint32_t round = (uint32_t)(kt / S);
                if (kt >= S && !mbar_wait_bounded(&empty[s], (round - 1) & 1, p.timeout_ns,
                                                  abort_flag, p.err))
                    break;
                mbar_arrive_expect_tx(&full[s], stage_bytes);
                if (kt == p.inject_skip_kt && blockIdx.x == 0) {
                    skipped = kt;         // fault injection: the stage never fills
                } else {
                    double* As = tiles + (size_t)s * stage_elems;
                    double* Bs = As + bm * bk;
                    tma_load_2d(As, &tmA, &full[s], (int32_t)(kt * bk), (int32_t)m0);
                    tma_load_2d(Bs, &tmB, &full[s], (int32_t)n0, (int32_t)(kt * bk));
                }
                issued = kt + 1;
            }
            // Before leaving, every copy this thread issued must have landed:
            // the last min(S, issued) stages are the only ones possibly in flight.
            for (int64_t kt = (issued > S ? issued - S : 0); kt < issued; ++kt) {
                if (kt == skipped) continue;
                const int s = (int)(kt % S);
                const uint32_t round = (uint32_t)(kt / S);
                mbar_wait_bounded(&full[s], round & 1, p.timeout_ns, nullptr, p.err, false);
            }
        }
        return;
    }

    // ---------------- consumers ----------------
    const int cw = warp - 1;
    const int wn_count = bn / (4 * TN);
    const int wm0 = (cw / wn_count) * 8 * TM, wn0 = (cw % wn_count) * 4 * TN;
    Acc<TM, TN> acc;
    acc.zero();
    for (int64_t kt = 0; kt < KT; ++kt) {
        const int s = (int)(kt % S);
        const uint32_t round = (uint32_t)(kt / S);
        if (!mbar_wait_bounded(&full[s], round & 1, p.timeout_ns, abort_flag, p.err)) return;
        const double* As = tiles + (size_t)s * stage_elems;
        const double* Bs = As + bm * bk;
        mma_stage<TM, TN>(As, Bs, bk, bn, wm0, wn0, lane, acc);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    epilogue<TM, TN>(acc, p.C, p.ldc, p.M, p.N, m0 + wm0, n0 + wn0, p.alpha, p.beta, p.vec2 != 0,
                     lane);
}

// Non-TMA variant: same tiles and MMAs, cp.async loads by all threads.
struct LdgParams {
    TileProblem prob;
    int bm, bn, bk;
    int tiles_m, tiles_n;
    int vec2;
};

template <int TM, int TN>
__global__ void __launch_bounds__(max_threads(TM, TN), 1) dgemm_ldg_kernel(LdgParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    int tmi, tni;
    tile_coords(blockIdx.x, p.tiles_m, p.tiles_n, tmi, tni);
    tile_ldg<TM, TN>(p.prob, (int64_t)tmi * p.bm, (int64_t)tni * p.bn, p.bm, p.bn, p.bk,
                     reinterpret_cast<double*>(smem_raw), p.vec2 != 0);
}

// C = beta*C (alpha == 0 or K == 0); beta == 0 writes zeros without reading C.
__global__ void scale_kernel(double* C, int64_t ldc, int64_t M, int64_t N, double beta) {
    const int64_t total = M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N, j = e - i * N;
        double* c = C + i * ldc + j;
        *c = (beta == 0.0) ? 0.0 : beta * *c;
    }
}

// ----------------------------------------------------------------------------
// Host side.
// ----------------------------------------------------------------------------
template <int TM, int TN>
static alp_status launch_tm_tn(const alp_config& cfg, int stages, bool use_tma, int64_t M,
                               int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                               const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                               cudaStream_t stream, int inject_skip_kt, int64_t grid_limit) {
    const int tiles_m = (int)((M + cfg.bm - 1) / cfg.bm);
    const int tiles_n = (int)((N + cfg.bn - 1) / cfg.bn);
    int64_t grid = (int64_t)tiles_m * tiles_n;
    if (grid_limit > 0 && grid > grid_limit) grid = grid_limit;   // tuner's one-wave proxy
    if (grid > 0x7fffffff) return ALP_ERR_UNSUPPORTED;
    const bool vec2 = ((reinterpret_cast<uintptr_t>(C) & 15) == 0) && (ldc % 2 == 0);
    if (use_tma) {
        CUtensorMap ta, tb;
        alp_status st = make_tmap_2d(&ta, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, A, (uint64_t)K,
                                     (uint64_t)M, (uint64_t)lda * 8, cfg.bk, cfg.bm,
                                     CU_TENSOR_MAP_SWIZZLE_NONE);
        if (st != ALP_OK) return st;
        st = make_tmap_2d(&tb, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, B, (uint64_t)N, (uint64_t)K,
                          (uint64_t)ldb * 8, cfg.bn, cfg.bk, CU_TENSOR_MAP_SWIZZLE_NONE);
        if (st != ALP_OK) return st;
        NativeParams p;
        p.M = M; p.N = N; p.K = K; p.alpha = alpha; p.beta = beta; p.C = C; p.ldc = ldc;
        p.bm = cfg.bm; p.bn = cfg.bn; p.bk = cfg.bk; p.stages = stages;
        p.tiles_m = tiles_m; p.tiles_n = tiles_n; p.vec2 = vec2 ? 1 : 0;
        p.timeout_ns = wait_timeout_ns(); p.err = device_error_word();
        p.inject_skip_kt = inject_skip_kt;
        const int smem = (int)(native_stage_bytes(cfg.bm, cfg.bn, cfg.bk) * stages + 16 * stages + 16);
        const int threads = native_threads(cfg.bm, cfg.bn, TM, TN);
        cudaError_t e = cudaFuncSetAttribute(dgemm_tma_kernel<TM, TN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return cuda_status(e);
        dgemm_tma_kernel<TM, TN><<<(unsigned)grid, threads, smem, stream>>>(ta, tb, p);
        return cuda_status(cudaGetLastError());
    }
    LdgParams p;
    p.prob.A = A; p.prob.B = B; p.prob.C = C; p.prob.lda = lda; p.prob.ldb = ldb; p.prob.ldc = ldc;
    p.prob.M = M; p.prob.N = N; p.prob.K = K; p.prob.alpha = alpha; p.prob.beta = beta;
    p.bm = cfg.bm; p.bn = cfg.bn; p.bk = cfg.bk; p.tiles_m = tiles_m; p.tiles_n = tiles_n;
    p.vec2 = vec2 ? 1 : 0;
    const int smem = (int)(native_stage_bytes(cfg.bm, cfg.bn, cfg.bk) * 2);
    if (smem > kSmemLimit) return ALP_ERR_UNSUPPORTED;
    const int threads = 32 * native_compute_warps(cfg.bm, cfg.bn, TM, TN);
    cudaError_t e = cudaFuncSetAttribute(dgemm_ldg_kernel<TM, TN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_status(e);
    dgemm_ldg_kernel<TM, TN><<<(unsigned)grid, threads, smem, stream>>>(p);
    return cuda_status(cudaGetLastError());
}

// out (C x R, row stride ldo) = X^T for a row-major R x C matrix X (row
// stride ldx): 32 x 32 tiles through shared memory, reads and writes along rows.
__global__ void transpose_kernel(const double* __restrict__ X, int64_t R, int64_t Cn, int64_t ldx,
                                 double* __restrict__ out, int64_t ldo) {
    __shared__ double t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (r < R && c < Cn) ? X[r * ldx + c] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (c < Cn && r < R) out[c * ldo + r] = t[threadIdx.x][i];
    }
}

alp_status native_transpose(const double* X, int64_t R, int64_t Cn, int64_t ldx, double* out,
                            int64_t ldo, cudaStream_t stream) {
    if (R == 0 || Cn == 0) return ALP_OK;
    const int64_t gy = (R + 31) / 32, gx = (Cn + 31) / 32;
    if (gy > 65535 || gx > 0x7fffffff) return ALP_ERR_UNSUPPORTED;
    transpose_kernel<<<dim3((unsigned)gx, (unsigned)gy), dim3(32, 8), 0, stream>>>(X, R, Cn, ldx,
                                                                                   out, ldo);
    return cuda_status(cudaGetLastError());
}

alp_status native_scale(int64_t M, int64_t N, double beta, double* C, int64_t ldc,
                        cudaStream_t stream) {
    const int64_t total = M * N;
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    scale_kernel<<<(unsigned)blocks, 256, 0, stream>>>(C, ldc, M, N, beta);
    return cuda_status(cudaGetLastError());
}

// Launches one GEMM with a validated config.  use_tma selects the TMA kernel
// (caller checked its alignment rules).
alp_status native_launch(const alp_config& cfg, bool use_tma, int64_t M, int64_t N, int64_t K,
                         double alpha, const double* A, int64_t lda, const double* B,
                         int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t stream,
                         int inject_skip_kt, int64_t grid_limit) {
    const int stages = native_stages(cfg.bm, cfg.bn, cfg.bk, cfg.stages);
#define ALP_NATIVE_CASE(a, b)                                                                     \
    if (cfg.tm == a && cfg.tn == b)                                                               \
        return launch_tm_tn<a, b>(cfg, stages, use_tma, M, N, K, alpha, A, lda, B, ldb, beta, C, \
                                  ldc, stream, inject_skip_kt, grid_limit);
    ALP_NATIVE_CASE(2, 2) ALP_NATIVE_CASE(2, 4) ALP_NATIVE_CASE(2, 8)
    ALP_NATIVE_CASE(4, 2) ALP_NATIVE_CASE(4, 4) ALP_NATIVE_CASE(4, 8)
    ALP_NATIVE_CASE(8, 2) ALP_NATIVE_CASE(8, 4) ALP_NATIVE_CASE(8, 8)
#undef ALP_NATIVE_CASE
    return ALP_ERR_INVALID_ARG;
}

// Blocks of this config that fit on one SM (0: cannot launch on this GPU).
// Failed queries are consumed so that no CUDA error is left pending.
int native_occupancy(const alp_config& cfg, bool use_tma) {
    const int stages = native_stages(cfg.bm, cfg.bn, cfg.bk, cfg.stages);
    const int64_t need = use_tma ? native_stage_bytes(cfg.bm, cfg.bn, cfg.bk) * stages + 16 * stages + 16
                                 : native_stage_bytes(cfg.bm, cfg.bn, cfg.bk) * 2;
    if (need > kSmemLimit) return 0;
    int n = 0;
#define ALP_OCC_CASE(a, b)                                                                        \
    if (cfg.tm == a && cfg.tn == b) {                                                             \
        const int smem = use_tma ? (int)(native_stage_bytes(cfg.bm, cfg.bn, cfg.bk) * stages +    \
                                         16 * stages + 16)                                        \
                                 : (int)(native_stage_bytes(cfg.bm, cfg.bn, cfg.bk) * 2);         \
        const int thr = use_tma ? native_threads(cfg.bm, cfg.bn, a, b)                            \
                                : 32 * native_compute_warps(cfg.bm, cfg.bn, a, b);                \
        if (use_tma) {                                                                            \
            cudaFuncSetAttribute(dgemm_tma_kernel<a, b>,                                          \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);              \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dgemm_tma_kernel<a, b>, thr, smem); \
        } else {                                                                                  \
            cudaFuncSetAttribute(dgemm_ldg_kernel<a, b>,                                          \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);              \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dgemm_ldg_kernel<a, b>, thr, smem); \
        }                                                                                         \
    }
    ALP_OCC_CASE(2, 2) ALP_OCC_CASE(2, 4) ALP_OCC_CASE(2, 8)
    ALP_OCC_CASE(4, 2) ALP_OCC_CASE(4, 4) ALP_OCC_CASE(4, 8)
    ALP_OCC_CASE(8, 2) ALP_OCC_CASE(8, 4) ALP_OCC_CASE(8, 8)
#undef ALP_OCC_CASE
    cudaGetLastError();
    return n;
}

}  // namespace alp
