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

// ---- TMEM drain: exact conversion of integer-valued f32 accumulators ----
//
// A chunk of digit products leaves in each accumulator an f32 integer f with
// |f| <= 2^24 (f32 holds every such integer, so the MMAs never rounded).  Its
// value enters a 32-bit running sum exactly, without a float-to-int
// conversion, in four exact f32 steps:
//   y = f + C, C = 1.5 * 2^25: y lies in [2^25, 2^26], where the f32 spacing
//        is 4, so y = C + h with h = f rounded to a multiple of 4 and the bit
//        pattern of y is bits(C) + h / 4;
//   h = y - C and r = f - h are exact (Sterbenz; |r| <= 2);
//   z = r + M, M = 1.5 * 2^23: bits(z) = bits(M) + r.
// So 4 bits(y) + bits(z) = (4 bits(C) + bits(M)) + f (mod 2^32): the sum of
// these over n chunks minus n * kChunkBias is the exact sum of the f.
constexpr uint32_t kChunkBias = 0x7C400000u;   // 4 * 0x4C400000 + 0x4B400000 mod 2^32

// 32 columns of this thread's TMEM lane: one load, one wait, the conversion
// above into a[0..31].  Load, wait and arithmetic form one asm block, so no
// value is used before the wait.
__device__ __forceinline__ void tmem_drain32_exact(uint32_t taddr, uint32_t* a) {
    asm volatile(
        "{\n"
        " .reg .b32 r<32>;\n"
        " tcgen05.ld.sync.aligned.32x32b.x32.b32 {r0,r1,r2,r3,r4,r5,r6,r7,r8,r9,r10,r11,r12,r13,r14,r15,r16,r17,r18,r19,r20,r21,r22,r23,r24,r25,r26,r27,r28,r29,r30,r31}, [%32];\n"
        " tcgen05.wait::ld.sync.aligned;\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r0, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r0, r0, h;\n"
        "   add.rn.f32 r0, r0, 0f4B400000;\n"
        "   mad.lo.u32 %0, t, 4, %0;\n"
        "   add.u32 %0, %0, r0; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r1, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r1, r1, h;\n"
        "   add.rn.f32 r1, r1, 0f4B400000;\n"
        "   mad.lo.u32 %1, t, 4, %1;\n"
        "   add.u32 %1, %1, r1; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r2, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r2, r2, h;\n"
        "   add.rn.f32 r2, r2, 0f4B400000;\n"
        "   mad.lo.u32 %2, t, 4, %2;\n"
        "   add.u32 %2, %2, r2; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r3, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r3, r3, h;\n"
        "   add.rn.f32 r3, r3, 0f4B400000;\n"
        "   mad.lo.u32 %3, t, 4, %3;\n"
        "   add.u32 %3, %3, r3; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r4, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r4, r4, h;\n"
        "   add.rn.f32 r4, r4, 0f4B400000;\n"
        "   mad.lo.u32 %4, t, 4, %4;\n"
        "   add.u32 %4, %4, r4; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r5, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r5, r5, h;\n"
        "   add.rn.f32 r5, r5, 0f4B400000;\n"
        "   mad.lo.u32 %5, t, 4, %5;\n"
        "   add.u32 %5, %5, r5; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r6, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r6, r6, h;\n"
        "   add.rn.f32 r6, r6, 0f4B400000;\n"
        "   mad.lo.u32 %6, t, 4, %6;\n"
        "   add.u32 %6, %6, r6; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r7, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r7, r7, h;\n"
        "   add.rn.f32 r7, r7, 0f4B400000;\n"
        "   mad.lo.u32 %7, t, 4, %7;\n"
        "   add.u32 %7, %7, r7; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r8, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r8, r8, h;\n"
        "   add.rn.f32 r8, r8, 0f4B400000;\n"
        "   mad.lo.u32 %8, t, 4, %8;\n"
        "   add.u32 %8, %8, r8; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r9, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r9, r9, h;\n"
        "   add.rn.f32 r9, r9, 0f4B400000;\n"
        "   mad.lo.u32 %9, t, 4, %9;\n"
        "   add.u32 %9, %9, r9; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r10, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r10, r10, h;\n"
        "   add.rn.f32 r10, r10, 0f4B400000;\n"
        "   mad.lo.u32 %10, t, 4, %10;\n"
        "   add.u32 %10, %10, r10; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r11, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r11, r11, h;\n"
        "   add.rn.f32 r11, r11, 0f4B400000;\n"
        "   mad.lo.u32 %11, t, 4, %11;\n"
        "   add.u32 %11, %11, r11; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r12, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r12, r12, h;\n"
        "   add.rn.f32 r12, r12, 0f4B400000;\n"
        "   mad.lo.u32 %12, t, 4, %12;\n"
        "   add.u32 %12, %12, r12; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r13, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r13, r13, h;\n"
        "   add.rn.f32 r13, r13, 0f4B400000;\n"
        "   mad.lo.u32 %13, t, 4, %13;\n"
        "   add.u32 %13, %13, r13; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r14, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r14, r14, h;\n"
        "   add.rn.f32 r14, r14, 0f4B400000;\n"
        "   mad.lo.u32 %14, t, 4, %14;\n"
        "   add.u32 %14, %14, r14; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r15, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r15, r15, h;\n"
        "   add.rn.f32 r15, r15, 0f4B400000;\n"
        "   mad.lo.u32 %15, t, 4, %15;\n"
        "   add.u32 %15, %15, r15; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r16, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r16, r16, h;\n"
        "   add.rn.f32 r16, r16, 0f4B400000;\n"
        "   mad.lo.u32 %16, t, 4, %16;\n"
        "   add.u32 %16, %16, r16; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r17, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r17, r17, h;\n"
        "   add.rn.f32 r17, r17, 0f4B400000;\n"
        "   mad.lo.u32 %17, t, 4, %17;\n"
        "   add.u32 %17, %17, r17; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r18, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r18, r18, h;\n"
        "   add.rn.f32 r18, r18, 0f4B400000;\n"
        "   mad.lo.u32 %18, t, 4, %18;\n"
        "   add.u32 %18, %18, r18; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r19, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r19, r19, h;\n"
        "   add.rn.f32 r19, r19, 0f4B400000;\n"
        "   mad.lo.u32 %19, t, 4, %19;\n"
        "   add.u32 %19, %19, r19; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r20, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r20, r20, h;\n"
        "   add.rn.f32 r20, r20, 0f4B400000;\n"
        "   mad.lo.u32 %20, t, 4, %20;\n"
        "   add.u32 %20, %20, r20; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r21, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r21, r21, h;\n"
        "   add.rn.f32 r21, r21, 0f4B400000;\n"
        "   mad.lo.u32 %21, t, 4, %21;\n"
        "   add.u32 %21, %21, r21; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r22, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r22, r22, h;\n"
        "   add.rn.f32 r22, r22, 0f4B400000;\n"
        "   mad.lo.u32 %22, t, 4, %22;\n"
        "   add.u32 %22, %22, r22; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r23, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r23, r23, h;\n"
        "   add.rn.f32 r23, r23, 0f4B400000;\n"
        "   mad.lo.u32 %23, t, 4, %23;\n"
        "   add.u32 %23, %23, r23; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r24, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r24, r24, h;\n"
        "   add.rn.f32 r24, r24, 0f4B400000;\n"
        "   mad.lo.u32 %24, t, 4, %24;\n"
        "   add.u32 %24, %24, r24; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r25, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r25, r25, h;\n"
        "   add.rn.f32 r25, r25, 0f4B400000;\n"
        "   mad.lo.u32 %25, t, 4, %25;\n"
        "   add.u32 %25, %25, r25; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r26, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r26, r26, h;\n"
        "   add.rn.f32 r26, r26, 0f4B400000;\n"
        "   mad.lo.u32 %26, t, 4, %26;\n"
        "   add.u32 %26, %26, r26; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r27, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r27, r27, h;\n"
        "   add.rn.f32 r27, r27, 0f4B400000;\n"
        "   mad.lo.u32 %27, t, 4, %27;\n"
        "   add.u32 %27, %27, r27; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r28, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r28, r28, h;\n"
        "   add.rn.f32 r28, r28, 0f4B400000;\n"
        "   mad.lo.u32 %28, t, 4, %28;\n"
        "   add.u32 %28, %28, r28; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r29, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r29, r29, h;\n"
        "   add.rn.f32 r29, r29, 0f4B400000;\n"
        "   mad.lo.u32 %29, t, 4, %29;\n"
        "   add.u32 %29, %29, r29; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r30, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r30, r30, h;\n"
        "   add.rn.f32 r30, r30, 0f4B400000;\n"
        "   mad.lo.u32 %30, t, 4, %30;\n"
        "   add.u32 %30, %30, r30; }\n"
        " { .reg .b32 t, h;\n"
        "   add.rn.f32 t, r31, 0f4C400000;\n"
        "   sub.rn.f32 h, t, 0f4C400000;\n"
        "   sub.rn.f32 r31, r31, h;\n"
        "   add.rn.f32 r31, r31, 0f4B400000;\n"
        "   mad.lo.u32 %31, t, 4, %31;\n"
        "   add.u32 %31, %31, r31; }\n"
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
