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
 * (bm+bn)*bk*8 bytes within 227 KiB of shared memory. */
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
 * kernel returns.  kt = -1 switches it off.  No copy is left in flight. */
alp_status alp_debug_inject_skip(int kt);

/* ---- FP64 peak probe ----------------------------------------------------- */

/* Measured FP64 throughput of this GPU: kind 0 = m16n8k4 DMMA chains (the
 * native kernel's instruction), kind 1 = scalar DFMA chains; blocks_per_sm x
 * SM-count blocks of `threads` threads, each warp/thread running 8 independent
 * chains for `iters` iterations.  One warm-up launch, one launch timed with
 * CUDA events on `stream` (synchronises it).  Result in TFLOP/s (2 per FMA). */
alp_status alp_probe_fp64_peak(int kind, int64_t iters, int blocks_per_sm, int threads,
                               double* out_tflops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ALP_EXT_H */
