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
