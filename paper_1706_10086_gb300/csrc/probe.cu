// FP64 peak probes: the denominators of the native kernel's roofline.  GB300
// (Blackwell Ultra) cut FP64 throughput far below earlier datacenter parts and
// no measured figure ships with the machine, so the library measures its own:
// long chains of independent FP64 MMAs of each shape the ISA offers (m16n8k4,
// the instruction the native kernel issues, m16n8k8 and m16n8k16) and of
// scalar DFMAs, on every SM, timed with CUDA events.
#include "alp_ext.h"
#include "alp_internal.cuh"

namespace alp {

constexpr int kChains = 8;   // independent accumulators per warp/thread (latency cover)

__global__ void probe_dmma_kernel(int64_t iters, double* sink) {
    double c[kChains][4];
    const double a0 = 1.0 + threadIdx.x * 1e-9, a1 = 1.0 - threadIdx.x * 1e-9;
    const double b0 = 1e-12;
#pragma unroll
    for (int i = 0; i < kChains; ++i)
#pragma unroll
        for (int r = 0; r < 4; ++r) c[i][r] = 0.0;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) dmma_16x8x4(c[i], a0, a1, b0);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
    if (s == 12345.0) sink[threadIdx.x] = s;   // never true; keeps the chains live
}

// The larger FP64 MMA shapes: m16n8k8 (A 4, B 2 registers per thread) and
// m16n8k16 (A 8, B 4), C/D 4 registers as for m16n8k4.
__device__ __forceinline__ void dmma_16x8x8(double (&c)[4], const double (&a)[4],
                                            const double (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(b[0]), "d"(b[1]));
}
__device__ __forceinline__ void dmma_16x8x16(double (&c)[4], const double (&a)[8],
                                             const double (&b)[4]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
        "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};"
        : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]),
          "d"(a[7]), "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

// KK = 8 or 16: chains of m16n8kKK DMMAs.
template <int KK>
__global__ void probe_dmma_wide_kernel(int64_t iters, double* sink) {
    double c[kChains][4];
    double a[KK / 2], b[KK / 4];
#pragma unroll
    for (int i = 0; i < KK / 2; ++i) a[i] = 1.0 + (threadIdx.x + i) * 1e-9;
#pragma unroll
    for (int i = 0; i < KK / 4; ++i) b[i] = 1e-12 * (i + 1);
#pragma unroll
    for (int i = 0; i < kChains; ++i)
#pragma unroll
        for (int r = 0; r < 4; ++r) c[i][r] = 0.0;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            if constexpr (KK == 8) dmma_16x8x8(c[i], a, b);
            else dmma_16x8x16(c[i], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
    if (s == 12345.0) sink[threadIdx.x] = s;   // never true; keeps the chains live
}

__global__ void probe_dfma_kernel(int64_t iters, double* sink) {
    double c[kChains];
    const double a = 1.0 + threadIdx.x * 1e-9, b = 1e-12;
#pragma unroll
    for (int i = 0; i < kChains; ++i) c[i] = (double)i;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) c[i] = __fma_rn(a, c[i], b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += c[i];
    if (s == 12345.0) sink[threadIdx.x] = s;
}

}  // namespace alp

using namespace alp;

extern "C" alp_status alp_probe_fp64_peak(int kind, int64_t iters, int blocks_per_sm,
                                          int threads, double* out_tflops, void* stream) {
    if (!out_tflops || iters <= 0 || blocks_per_sm <= 0 || threads <= 0 || threads > 1024 ||
        threads % 32 || kind < 0 || kind > 3)
        return ALP_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int blocks = device_sm_count() * blocks_per_sm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return ALP_ERR_CUDA;
    double flops;
    // warm-up launch, then the timed one
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) cudaEventRecord(e0, s);
        if (kind == 0)
            probe_dmma_kernel<<<blocks, threads, 0, s>>>(iters, nullptr);
        else if (kind == 1)
            probe_dfma_kernel<<<blocks, threads, 0, s>>>(iters, nullptr);
        else if (kind == 2)
            probe_dmma_wide_kernel<8><<<blocks, threads, 0, s>>>(iters, nullptr);
        else
            probe_dmma_wide_kernel<16><<<blocks, threads, 0, s>>>(iters, nullptr);
        if (cudaGetLastError() != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return ALP_ERR_UNSUPPORTED;   // e.g. too many registers for `threads`
        }
    }
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return ALP_ERR_CUDA;
    if (kind == 1)
        flops = 2.0 * kChains * (double)iters * blocks * threads;
    else   // per warp per DMMA: 16*8*k multiply-adds, k = 4, 8, 16
        flops = 2.0 * 16 * 8 * (kind == 0 ? 4 : kind == 2 ? 8 : 16) * kChains * (double)iters *
                blocks * (threads / 32);
    *out_tflops = flops / (ms * 1e-3) / 1e12;
    return ALP_OK;
}
