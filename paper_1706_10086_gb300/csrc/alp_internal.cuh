// Internal helpers shared by the library's translation units: status plumbing,
// the device error word, bounded mbarrier waits, TMA and tcgen05 wrappers
// (inline PTX for sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "alp.h"

namespace alp {

// ----------------------------------------------------------------------------
// Device error word.  Kernels never trap: a failed check or an expired wait
// records a code in the word (first writer wins) and the kernel returns.  Every
// kernel receives the word's address; abi.cu owns one word per device.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void set_device_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// Host-side knobs (defined in abi.cu).
int* device_error_word();             // address of the current device's word
uint64_t wait_timeout_ns();           // limit of every device-side wait
int device_sm_count();
alp_status cuda_status(cudaError_t e);
int inject_skip_kt();                 // test hook of the timeout path (-1: off)

// ----------------------------------------------------------------------------
// Time and barriers.
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile(
        "{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
            smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of `bar` to complete.  Gives up after `limit_ns`
// (or at once when *abort is set by another role of the block, or when some
// block of any launch has already recorded ALP_ERR_TIMEOUT, so that a broken
// launch ends after one limit rather than one limit per wave), records
// ALP_ERR_TIMEOUT and returns false; the caller then leaves its loop.
// Waits that make sure a block's own copies or MMAs have finished before it
// frees shared memory or TMEM pass follow_global = false: they always wait for
// the barrier itself (or their own limit).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns, volatile int* abort,
                                                  int* err, bool follow_global = true) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort && *abort) return false;
        // the global error word and the clock every 64 polls: a global load in
        // every poll would delay noticing the phase by its latency
        if ((i & 63u) != 0) continue;
        if (follow_global && err && *reinterpret_cast<volatile int*>(err) == ALP_ERR_TIMEOUT) {
            if (abort) *abort = 1;
            return false;
        }
        if (globaltimer() - t0 > limit_ns) {
            set_device_error(err, ALP_ERR_TIMEOUT);
            if (abort) *abort = 1;
            return false;
        }
    }
}

// ----------------------------------------------------------------------------
// TMA (cp.async.bulk.tensor), 2-D tiles, completion on an mbarrier.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map,
                                            uint64_t* bar, int32_t x, int32_t y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Untiled bulk copy of `bytes` from global to this CTA's shared memory, both
// addresses 16-byte aligned and bytes a multiple of 16, completing on `bar`
// (complete_tx).
__device__ __forceinline__ void bulk_load(void* smem_dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ----------------------------------------------------------------------------
// FP64 DMMA: D(16x8) += A(16x4, row) * B(4x8, col), sm_90+ shape.
// Fragment ownership (lane = 4*g + t):  a0 = A[g][t], a1 = A[g+8][t];
// b0 = B[t][g];  c0,c1 = C[g][2t..2t+1], c2,c3 = C[g+8][2t..2t+1].
// ----------------------------------------------------------------------------
__device__ __forceinline__ void dmma_16x8x4(double (&c)[4], double a0, double a1, double b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%0,%1,%2,%3};"
        : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
        : "d"(a0), "d"(a1), "d"(b0));
}

// Host helpers (abi.cu).
alp_status make_tmap_2d(CUtensorMap* map, CUtensorMapDataType dtype, int elem_bytes,
                        const void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                        uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz);

}  // namespace alp
