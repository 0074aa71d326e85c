/*
 * alp_ext.h -- companion entry points of alp.h: tile-configuration queries
 * (host only, no GPU needed), device-wait limits and the test hook that
 * exercises them, the FP64 peak probe, and the cost model's kernels.
 * Same conventions as alp.h (device pointers owned by the caller, streams as
 * void*, status codes, no exceptions).
 */
#ifndef ALP_EXT_H
#define ALP_EXT_H

#include "alp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- tile configurations (host logic) ---------------------------------- */

/* 1 if cfg is a valid config of `path`, else 0.  Native rules: bm, bn in
 * {64,128,256}; bk in {16,32,64}; tm, tn in {2,4,8}; one producer warp plus
 * (bm/(8 tm)) * (bn/(4 tn)) compute warps within the per-(tm,tn) thread cap
 * that keeps the register tile resident; at least 2 stages of
 * (bm+bn)*bk*8 bytes within 227 KiB of shared memory.  Emulated path:
 * {128, 256, 64, 1, 0, group} (one block per 128 x 256 tile), or
 * {256, 256, 64, 2, 0, group} (CTA pairs whose tcgen05 MMAs span both SMs on
 * a 256 x 256 tile; the default), and group in {1, 2, 4, 8, 16, 32}
 * (tile-rows per raster group). */
int alp_config_valid(const alp_config* cfg, alp_path path);

/* Shared-memory bytes of the A and B tiles of all stages: stages*(bm+bn)*bk*8
 * (stages = 0 means the automatic count).  With bm = bn = bk = T and one stage
 * this is the tile cache model K(S,T) = 2 T^2 S of Eq. 3 for S = 8 bytes. */
int64_t alp_config_smem_bytes(const alp_config* cfg);

/* Threads per block of the native TMA kernel for cfg. */
int alp_config_threads(const alp_config* cfg);

/* Number of valid configs of `path`, and the idx-th of them in sweep order
 * (bm, bn, bk, tm, tn ascending, automatic stages). */
int alp_config_count(alp_path path);
alp_status alp_config_at(alp_path path, int idx, alp_config* out);

/* ---- device-side waits -------------------------------------------------- */

/* Limit of every device-side wait (default 4000 ms or env ALP_WAIT_TIMEOUT_MS). */
alp_status alp_set_wait_timeout_ms(double ms);

/* Test hook for the timeout path: while kt >= 0, the producer warp of block 0
 * of each native TMA GEMM arms stage kt's barrier but issues no copy into it,
 * so that the consumers' wait runs out, ALP_ERR_TIMEOUT is recorded and the
 * kernel returns.  The emulated path's tensor-core kernel does the same with
 * its kt-th pipeline stage (counted over all jobs of block 0; for CTA pairs
 * block 0 of the first pair skips its half, so the pair's stage never fills).
 * kt = -1 switches it off.  No copy is left in flight. */
alp_status alp_debug_inject_skip(int kt);

/* ---- autotuner helpers --------------------------------------------------- */

/* Time of one config for (M, N, K) on `path`, in ms: the best of `runs`
 * CUDA-event-timed launches after one warm-up.  use_proxy = 1 estimates (the
 * estimate alp_tune records): native, one wave of blocks with K capped at 256,
 * scaled by the waves and by K / 256; emulated, the tensor-core stage on the
 * whole grid with K capped at 2048 (env ALP_TUNE_PROXY_K_EMUL), scaled by
 * K / cap.  use_proxy = 0 times the whole problem (for the emulated path, its
 * tensor-core stage).  Allocates its own scratch. */
alp_status alp_tune_time_config(int64_t M, int64_t N, int64_t K, alp_path path,
                                const alp_config* cfg, int use_proxy, int runs, double* est_ms);
/* Puts cfg into the tuned cache for (M, N, K, path) (what alp_tune(EXHAUSTIVE)
 * does with its winner), and empties the cache. */
alp_status alp_tune_set_cached(int64_t M, int64_t N, int64_t K, alp_path path,
                               const alp_config* cfg);
alp_status alp_tune_clear_cache(void);

/* ---- learned cost model (FP32 MLP 7 -> 64 -> 64 -> C, ReLU) -------------- */
/* Parameters: one float array W1[64][7], b1[64], W2[64][64], b2[64], W3[C][64],
 * b3[C] (alp_mlp_param_count(C) floats).  C = alp_config_count(NATIVE) +
 * alp_config_count(EMUL): outputs 0.. are the native configs in sweep order,
 * then the emulated path's.  All arrays are device memory unless noted. */
int64_t alp_mlp_param_count(int C);
/* X[i][0..6] = (log2 M, log2 N, log2 K, log2 M/N, log2 N/K, log2 M/K, path)
 * for path = 0 (native) or 1 (emulated), minus mean and divided by std when
 * both are given (7 floats each). */
alp_status alp_mlp_features(int64_t count, const int64_t* dM, const int64_t* dN,
                            const int64_t* dK, const int32_t* dpath, const float* mean,
                            const float* std, float* X, void* stream);
/* Per-feature mean and standard deviation of X (count x 7), for standardising. */
alp_status alp_mlp_feature_stats(int64_t count, const float* X, float* mean, float* std,
                                 void* stream);
/* Y (B x C) = forward(params, X (B x 7)); cache (B x 128) keeps the
 * pre-activations for alp_mlp_backward. */
alp_status alp_mlp_forward(const float* params, int C, const float* X, int64_t B, float* Y,
                           float* cache, void* stream);
/* Gradients (alp_mlp_param_count(C) floats) of the masked mean squared error
 * L = sum Mask (Y - T)^2 / sum Mask over B x C, from a forward pass's Y and
 * cache; loss_out[0] = L, loss_out[1] = sum Mask; work: B * (C + 128) floats. */
alp_status alp_mlp_backward(const float* params, int C, const float* X, int64_t B,
                            const float* cache, const float* Y, const float* T,
                            const float* Mask, float* grads, float* work, float* loss_out,
                            void* stream);
/* One Adam step (bias-corrected, step counts from 1) over n parameters. */
alp_status alp_mlp_adam(float* params, const float* grads, float* m, float* v, int64_t n,
                        int step, float lr, float beta1, float beta2, float eps, void* stream);
/* Installs a trained model (HOST arrays: params, 7-float mean and std) for
 * alp_tune(PREDICT) and for GEMM calls with cfg == NULL that miss the tuned
 * cache (the prediction runs the forward kernel once per new shape, then it
 * is cached); unload removes it. */
alp_status alp_tune_load_model(const float* host_params, int C, const float* host_mean,
                               const float* host_std);
alp_status alp_tune_unload_model(void);

/* ---- batched GEMM: size classes and CUDA graph -------------------------- */

/* Size class of a problem in alp_gemm_batched_varsize: 3 * r + c with
 * r = 0, 1, 2 for M <= 32, <= 64, larger and c likewise from N. */
int alp_batched_class_of(int64_t M, int64_t N);

/* Tile (bm x bn, K step bk) used for the problems of class `cls` (0..8):
 * bm, bn in {32, 64, 128}, bk in {16, 32, 64}; each tile runs on 8 warps with
 * a (bm/16) x (bn/16) register tile per thread.  Defaults: bm, bn = 32, 64,
 * 128 by class, bk = 32 for classes with a 32-wide side, else 16.  Process-wide
 * setting, read when a batched call is issued (or captured). */
alp_status alp_batched_set_class_config(int cls, int bm, int bn, int bk);
alp_status alp_batched_get_class_config(int cls, int* bm, int* bn, int* bk);

/* Captures one alp_gemm_batched_varsize call (same arguments, stream
 * omitted) into a CUDA graph and instantiates it; *graph_out receives an
 * opaque handle.  Launching the handle replays the plan and the persistent
 * kernel on `stream`, reading the device arrays as they are at launch time
 * (the pointers are fixed at capture; the grid is sized from hM/hN at capture
 * and stays correct for any sizes).  Destroy with alp_batched_graph_destroy. */
alp_status alp_batched_graph_create(int64_t count, const int64_t* dM, const int64_t* dN,
                                    const int64_t* dK, const double* dalpha,
                                    const double* const* dA, const int64_t* dlda,
                                    const double* const* dB, const int64_t* dldb,
                                    const double* dbeta, double* const* dC,
                                    const int64_t* dldc, const int64_t* hM,
                                    const int64_t* hN, const int64_t* hK, void* workspace,
                                    size_t workspace_bytes, void** graph_out);
alp_status alp_batched_graph_launch(void* graph, void* stream);
alp_status alp_batched_graph_destroy(void* graph);

/* Same computation as alp_gemm_batched_varsize (same arguments minus the
 * workspace), for callers that cannot allocate device memory where they issue
 * the GEMM: frameworks whose device memory belongs to their own pool
 * allocator, and real-time or long-running loops that must not enter the
 * allocator (cudaMalloc / cudaFree take locks and may synchronise the device).
 * The paper has no counterpart; this is an interface convenience.
 * The persistent kernel's work list lives in a 1 MiB array compiled into the
 * library (held on every GPU that loads it until the process exits), so
 * count is limited to about 65,000 problems: larger batches return
 * ALP_ERR_WORKSPACE and must use alp_gemm_batched_varsize.  Nothing is
 * allocated, by this call or by the library's one-time set-up.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and the SM count; make that first call before any stream capture.
 * All calls share the one array and each call rewrites it completely, so no
 * clearing is needed between calls, but two calls whose kernels overlap on
 * the GPU (e.g. on different streams without ordering) race on it. */
alp_status alp_gemm_batched_varsize_noalloc(int64_t count, const int64_t* dM, const int64_t* dN,
                                            const int64_t* dK, const double* dalpha,
                                            const double* const* dA, const int64_t* dlda,
                                            const double* const* dB, const int64_t* dldb,
                                            const double* dbeta, double* const* dC,
                                            const int64_t* dldc, const int64_t* hM,
                                            const int64_t* hN, const int64_t* hK, void* stream);

/* ---- emulated path: launch shape -------------------------------------------- */

/* Host-only query (no GPU needed): how alp_emul_slice_products cuts a launch
 * of `tiles` tiles with `nslices` slices on `sms` SMs (for CTA pairs: pair
 * tiles on sms / 2 pairs).  Blocks [0, *n_full) take whole tiles; each remaining
 * tile (the last, partial wave) is taken by *pieces blocks, piece i computing
 * the group sums S^t for t = t_lo[i]..t_hi[i] (arrays of 8).  The cut is the
 * contiguous one whose largest piece (in digit pairs of the kind's scheme:
 * group t holds t-1 pairs, or 2 when it is the trimmed last group) is
 * smallest, with at most
 * min(sms / r, nslices, 8) pieces for r tiles in the last wave.  Splitting the
 * groups changes no result: each group sum is exact and written once. */
alp_status alp_emul_tail_split(int tiles, int nslices, alp_slice_kind kind, int sms, int* n_full,
                               int* pieces, int* t_lo, int* t_hi);

/* ---- host-resident operands ---------------------------------------------- */

/* Whether kernels on the current device may read and write host memory
 * through the host's own page tables (a Grace host over NVLink-C2C): *pageable
 * = 1 when any host pointer (pageable or pinned) is valid in a kernel,
 * *host_page_tables = 1 when that access uses the host's page tables (no
 * migration).  When *pageable is 1, the emulated GEMMs accept host pointers
 * for A, B and C: the exponent scans and splits read A and B where they are
 * and the recombination writes C there (the workspace stays on the device,
 * the tensor-core stage reads only it).  The native GEMM's TMA loads need
 * device memory.  Host-only query. */
alp_status alp_host_access(int* pageable, int* host_page_tables);

/* ---- FP64 peak probe ----------------------------------------------------- */

/* Measured FP64 throughput of this GPU: kind 0 = m16n8k4 DMMA chains (the
 * native kernel's instruction), kind 1 = scalar DFMA chains, kind 2 = m16n8k8
 * DMMA chains, kind 3 = m16n8k16 DMMA chains; blocks_per_sm x
 * SM-count blocks of `threads` threads, each warp/thread running 8 independent
 * chains for `iters` iterations.  One warm-up launch, one launch timed with
 * CUDA events on `stream` (synchronises it).  Result in TFLOP/s (2 per FMA). */
alp_status alp_probe_fp64_peak(int kind, int64_t iters, int blocks_per_sm, int threads,
                               double* out_tflops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ALP_EXT_H */
