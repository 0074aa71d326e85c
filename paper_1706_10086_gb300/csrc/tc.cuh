// tcgen05 (5th-generation tensor core) and 3-D TMA wrappers, inline PTX for
// sm_103a.  Conventions follow the PTX ISA for tcgen05:
//  * TMEM addresses: bits 31..16 lane, bits 15..0 column.
//  * Shared-memory matrix descriptor (64 bit): start address >> 4 in bits
//    0..13, leading-dimension byte offset >> 4 in 16..29, stride-dimension
//    byte offset >> 4 in 32..45, descriptor version 1 in 46..47, base offset
//    in 49..51, layout (swizzle) type in 61..63 (2 = 128-byte swizzle).
//  * Instruction descriptor of kind::f16 (32 bit): D format in 4..5 (1 = f32),
//    A format in 7..9 and B format in 10..12 (1 = bf16), A/B major in 15/16
//    (0 = K-major), N >> 3 in 17..22, M >> 4 in 24..28.
#pragma once

#include "alp_internal.cuh"

namespace alp {

__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* map,
                                            uint64_t* bar, int32_t x, int32_t y, int32_t z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Same, multicast to the CTAs of the cluster in `mask`: the tile lands at the
// same shared-memory offset in each and completes bytes on the mbarrier at
// the same offset in each.
__device__ __forceinline__ void tma_load_3d_multicast(void* smem_dst, const CUtensorMap* map,
                                                      uint64_t* bar, int32_t x, int32_t y,
                                                      int32_t z, uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        ".multicast::cluster [%0], [%1, {%3, %4, %5}], [%2], %6;" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z),
        "h"(mask)
        : "memory");
}

// ---- clusters ----
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// All threads of all CTAs of the cluster.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

// ---- TMEM allocation (one warp executes each) ----
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// ---- ordering of tcgen05 operations across thread synchronisation ----
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- MMA: D[tmem] (+)= A[smem] * B[smem]^T, bf16 inputs, f32 accumulation ----
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives once on `bar` when every tcgen05 operation this thread issued so far
// has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Arrives once on the mbarrier at `bar`'s offset in every CTA of `mask` when
// the thread's prior tcgen05 operations have completed.
__device__ __forceinline__ void umma_commit_multicast(uint64_t* bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)),
        "h"(mask)
        : "memory");
}

// ---- TMEM -> registers: 32 lanes x 16 columns of 32 bit (one row per thread) ----
__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_32x32b_x8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr));
}
// Loads 8 columns of this thread's TMEM lane (f32 holding integers |x| <= 2^22),
// waits for them, and adds each one's pattern (x + 1.5 * 2^23) into acc: the
// load, the wait and the adds form one asm block, so no value is used before
// the wait and no loaded register outlives it.
__device__ __forceinline__ void tmem_drain8_magic(uint32_t taddr, uint32_t& a0, uint32_t& a1,
                                                  uint32_t& a2, uint32_t& a3, uint32_t& a4,
                                                  uint32_t& a5, uint32_t& a6, uint32_t& a7) {
    asm volatile(
        "{\n"
        " .reg .b32 r<8>;\n"
        " tcgen05.ld.sync.aligned.32x32b.x8.b32 {r0,r1,r2,r3,r4,r5,r6,r7}, [%8];\n"
        " tcgen05.wait::ld.sync.aligned;\n"
        " add.rn.f32 r0, r0, 0f4B400000;\n add.rn.f32 r1, r1, 0f4B400000;\n"
        " add.rn.f32 r2, r2, 0f4B400000;\n add.rn.f32 r3, r3, 0f4B400000;\n"
        " add.rn.f32 r4, r4, 0f4B400000;\n add.rn.f32 r5, r5, 0f4B400000;\n"
        " add.rn.f32 r6, r6, 0f4B400000;\n add.rn.f32 r7, r7, 0f4B400000;\n"
        " add.u32 %0, %0, r0;\n add.u32 %1, %1, r1;\n add.u32 %2, %2, r2;\n"
        " add.u32 %3, %3, r3;\n add.u32 %4, %4, r4;\n add.u32 %5, %5, r5;\n"
        " add.u32 %6, %6, r6;\n add.u32 %7, %7, r7;\n"
        "}\n"
        : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3), "+r"(a4), "+r"(a5), "+r"(a6), "+r"(a7)
        : "r"(taddr)
        : "memory");
}

// 32 columns per call: one load, one wait, 32 exact adds (fewer round trips
// to TMEM than four 8-column calls).
__device__ __forceinline__ void tmem_drain32_magic(uint32_t taddr, uint32_t* a) {
    asm volatile(
        "{\n"
        " .reg .b32 r<32>;\n"
        " tcgen05.ld.sync.aligned.32x32b.x32.b32 {r0,r1,r2,r3,r4,r5,r6,r7,r8,r9,r10,r11,r12,r13,r14,r15,r16,r17,r18,r19,r20,r21,r22,r23,r24,r25,r26,r27,r28,r29,r30,r31}, [%32];\n"
        " tcgen05.wait::ld.sync.aligned;\n"
        " add.rn.f32 r0, r0, 0f4B400000;\n add.rn.f32 r1, r1, 0f4B400000;\n add.rn.f32 r2, r2, 0f4B400000;\n add.rn.f32 r3, r3, 0f4B400000;\n add.rn.f32 r4, r4, 0f4B400000;\n add.rn.f32 r5, r5, 0f4B400000;\n add.rn.f32 r6, r6, 0f4B400000;\n add.rn.f32 r7, r7, 0f4B400000;\n add.rn.f32 r8, r8, 0f4B400000;\n add.rn.f32 r9, r9, 0f4B400000;\n add.rn.f32 r10, r10, 0f4B400000;\n add.rn.f32 r11, r11, 0f4B400000;\n add.rn.f32 r12, r12, 0f4B400000;\n add.rn.f32 r13, r13, 0f4B400000;\n add.rn.f32 r14, r14, 0f4B400000;\n add.rn.f32 r15, r15, 0f4B400000;\n add.rn.f32 r16, r16, 0f4B400000;\n add.rn.f32 r17, r17, 0f4B400000;\n add.rn.f32 r18, r18, 0f4B400000;\n add.rn.f32 r19, r19, 0f4B400000;\n add.rn.f32 r20, r20, 0f4B400000;\n add.rn.f32 r21, r21, 0f4B400000;\n add.rn.f32 r22, r22, 0f4B400000;\n add.rn.f32 r23, r23, 0f4B400000;\n add.rn.f32 r24, r24, 0f4B400000;\n add.rn.f32 r25, r25, 0f4B400000;\n add.rn.f32 r26, r26, 0f4B400000;\n add.rn.f32 r27, r27, 0f4B400000;\n add.rn.f32 r28, r28, 0f4B400000;\n add.rn.f32 r29, r29, 0f4B400000;\n add.rn.f32 r30, r30, 0f4B400000;\n add.rn.f32 r31, r31, 0f4B400000;\n"
        " add.u32 %0, %0, r0;\n add.u32 %1, %1, r1;\n add.u32 %2, %2, r2;\n add.u32 %3, %3, r3;\n add.u32 %4, %4, r4;\n add.u32 %5, %5, r5;\n add.u32 %6, %6, r6;\n add.u32 %7, %7, r7;\n add.u32 %8, %8, r8;\n add.u32 %9, %9, r9;\n add.u32 %10, %10, r10;\n add.u32 %11, %11, r11;\n add.u32 %12, %12, r12;\n add.u32 %13, %13, r13;\n add.u32 %14, %14, r14;\n add.u32 %15, %15, r15;\n add.u32 %16, %16, r16;\n add.u32 %17, %17, r17;\n add.u32 %18, %18, r18;\n add.u32 %19, %19, r19;\n add.u32 %20, %20, r20;\n add.u32 %21, %21, r21;\n add.u32 %22, %22, r22;\n add.u32 %23, %23, r23;\n add.u32 %24, %24, r24;\n add.u32 %25, %25, r25;\n add.u32 %26, %26, r26;\n add.u32 %27, %27, r27;\n add.u32 %28, %28, r28;\n add.u32 %29, %29, r29;\n add.u32 %30, %30, r30;\n add.u32 %31, %31, r31;\n"
        "}\n"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]), "+r"(a[16]), "+r"(a[17]), "+r"(a[18]), "+r"(a[19]), "+r"(a[20]), "+r"(a[21]), "+r"(a[22]), "+r"(a[23]), "+r"(a[24]), "+r"(a[25]), "+r"(a[26]), "+r"(a[27]), "+r"(a[28]), "+r"(a[29]), "+r"(a[30]), "+r"(a[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Descriptor of a K-major operand tile stored by TMA with 128-byte swizzle:
// rows of 64 bf16 (128 bytes), 8-row core groups 1024 bytes apart.  The tile
// base must be 1024-byte aligned; advancing K by 16 elements inside the
// 128-byte row adds 32 bytes to the start address.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4)                        // D: f32
           | (1u << 7)                      // A: bf16
           | (1u << 10)                     // B: bf16
           | ((uint32_t)(N >> 3) << 17)     // N
           | ((uint32_t)(M >> 4) << 24);    // M
}

}  // namespace alp
