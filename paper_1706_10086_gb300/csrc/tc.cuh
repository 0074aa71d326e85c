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

// ---- CTA pairs (tcgen05 .cta_group::2): one MMA spans the SMs of a 2-CTA
// cluster.  A is split by rows and B by columns between the two CTAs (each
// holds its halves at the same shared-memory offsets), D by rows (each CTA's
// TMEM holds its 128 rows).  One thread of the even CTA issues the MMAs. ----

// The shared::cluster address of `p`'s counterpart in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

// TMA load into this CTA's shared memory that completes its bytes on an
// mbarrier of either CTA of the pair (`bar_cluster`, a shared::cluster address).
__device__ __forceinline__ void tma_load_3d_pair(void* smem_dst, const CUtensorMap* map,
                                                 uint32_t bar_cluster, int32_t x, int32_t y,
                                                 int32_t z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Arrive (release, cluster scope) on an mbarrier of another CTA of the cluster.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster)
                 : "memory");
}
// `count` arrivals at once on an mbarrier of another block of the cluster.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster, uint32_t count) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(
                     bar_cluster),
                 "r"(count)
                 : "memory");
}

// TMEM allocation for a CTA pair: one warp of each CTA executes each call.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// D[tmem of both CTAs] (+)= A * B^T for the pair (M = 256 in the descriptor).
__device__ __forceinline__ void umma_bf16_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                               uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives once on the mbarrier at `bar`'s offset in each CTA of `mask` when
// the pair MMAs this thread issued so far have completed.
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)),
        "h"(mask)
        : "memory");
}

// ---- TMEM drain ----
//
// A chunk of digit products leaves in each accumulator an f32 integer f with
// |f| <= 2^24 (f32 holds every such integer, so the MMAs never rounded);
// cvt.rzi.s32.f32 returns it exactly, and it enters a 32-bit running sum.
// (Two instructions per value: a conversion through four exact f32 additions
// issued three times as many and slowed the MMAs measurably.)

// 32 columns of this thread's TMEM lane: one load, one wait, the conversions
// and adds into a[0..31].  Load, wait and arithmetic form one asm block, so no
// value is used before the wait.
__device__ __forceinline__ void tmem_drain32_cvt(uint32_t taddr, uint32_t* a) {
    asm volatile(
        "{\n"
        " .reg .b32 r<32>;\n"
        " tcgen05.ld.sync.aligned.32x32b.x32.b32 {r0,r1,r2,r3,r4,r5,r6,r7,r8,r9,r10,r11,r12,r13,r14,r15,r16,r17,r18,r19,r20,r21,r22,r23,r24,r25,r26,r27,r28,r29,r30,r31}, [%32];\n"
        " tcgen05.wait::ld.sync.aligned;\n"
        " cvt.rzi.s32.f32 r0, r0;\n"
        " add.u32 %0, %0, r0;\n"
        " cvt.rzi.s32.f32 r1, r1;\n"
        " add.u32 %1, %1, r1;\n"
        " cvt.rzi.s32.f32 r2, r2;\n"
        " add.u32 %2, %2, r2;\n"
        " cvt.rzi.s32.f32 r3, r3;\n"
        " add.u32 %3, %3, r3;\n"
        " cvt.rzi.s32.f32 r4, r4;\n"
        " add.u32 %4, %4, r4;\n"
        " cvt.rzi.s32.f32 r5, r5;\n"
        " add.u32 %5, %5, r5;\n"
        " cvt.rzi.s32.f32 r6, r6;\n"
        " add.u32 %6, %6, r6;\n"
        " cvt.rzi.s32.f32 r7, r7;\n"
        " add.u32 %7, %7, r7;\n"
        " cvt.rzi.s32.f32 r8, r8;\n"
        " add.u32 %8, %8, r8;\n"
        " cvt.rzi.s32.f32 r9, r9;\n"
        " add.u32 %9, %9, r9;\n"
        " cvt.rzi.s32.f32 r10, r10;\n"
        " add.u32 %10, %10, r10;\n"
        " cvt.rzi.s32.f32 r11, r11;\n"
        " add.u32 %11, %11, r11;\n"
        " cvt.rzi.s32.f32 r12, r12;\n"
        " add.u32 %12, %12, r12;\n"
        " cvt.rzi.s32.f32 r13, r13;\n"
        " add.u32 %13, %13, r13;\n"
        " cvt.rzi.s32.f32 r14, r14;\n"
        " add.u32 %14, %14, r14;\n"
        " cvt.rzi.s32.f32 r15, r15;\n"
        " add.u32 %15, %15, r15;\n"
        " cvt.rzi.s32.f32 r16, r16;\n"
        " add.u32 %16, %16, r16;\n"
        " cvt.rzi.s32.f32 r17, r17;\n"
        " add.u32 %17, %17, r17;\n"
        " cvt.rzi.s32.f32 r18, r18;\n"
        " add.u32 %18, %18, r18;\n"
        " cvt.rzi.s32.f32 r19, r19;\n"
        " add.u32 %19, %19, r19;\n"
        " cvt.rzi.s32.f32 r20, r20;\n"
        " add.u32 %20, %20, r20;\n"
        " cvt.rzi.s32.f32 r21, r21;\n"
        " add.u32 %21, %21, r21;\n"
        " cvt.rzi.s32.f32 r22, r22;\n"
        " add.u32 %22, %22, r22;\n"
        " cvt.rzi.s32.f32 r23, r23;\n"
        " add.u32 %23, %23, r23;\n"
        " cvt.rzi.s32.f32 r24, r24;\n"
        " add.u32 %24, %24, r24;\n"
        " cvt.rzi.s32.f32 r25, r25;\n"
        " add.u32 %25, %25, r25;\n"
        " cvt.rzi.s32.f32 r26, r26;\n"
        " add.u32 %26, %26, r26;\n"
        " cvt.rzi.s32.f32 r27, r27;\n"
        " add.u32 %27, %27, r27;\n"
        " cvt.rzi.s32.f32 r28, r28;\n"
        " add.u32 %28, %28, r28;\n"
        " cvt.rzi.s32.f32 r29, r29;\n"
        " add.u32 %29, %29, r29;\n"
        " cvt.rzi.s32.f32 r30, r30;\n"
        " add.u32 %30, %30, r30;\n"
        " cvt.rzi.s32.f32 r31, r31;\n"
        " add.u32 %31, %31, r31;\n"
        "}\n"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]), "+r"(a[16]), "+r"(a[17]), "+r"(a[18]), "+r"(a[19]), "+r"(a[20]), "+r"(a[21]), "+r"(a[22]), "+r"(a[23]), "+r"(a[24]), "+r"(a[25]), "+r"(a[26]), "+r"(a[27]), "+r"(a[28]), "+r"(a[29]), "+r"(a[30]), "+r"(a[31])
        : "r"(taddr)
        : "memory");
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
