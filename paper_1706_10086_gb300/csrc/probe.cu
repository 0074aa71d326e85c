// FP64 peak probes: the denominators of the native kernel's roofline.  GB300
// (Blackwell Ultra) cut FP64 throughput far below earlier datacenter parts and
// no measured figure ships with the machine, so the library measures its own:
// long chains of independent m16n8k4 DMMAs (the instruction the native kernel
// issues) and of scalar DFMAs, on every SM, timed with CUDA events.
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
        threads % 32)
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
        else
            probe_dfma_kernel<<<blocks, threads, 0, s>>>(iters, nullptr);
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
    if (kind == 0)   // per warp per DMMA: 16*8*4 multiply-adds
        flops = 2.0 * 16 * 8 * 4 * kChains * (double)iters * blocks * (threads / 32);
    else
        flops = 2.0 * kChains * (double)iters * blocks * threads;
    *out_tflops = flops / (ms * 1e-3) / 1e12;
    return ALP_OK;
}
