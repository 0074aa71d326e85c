// Learned tile-config cost model: an FP32 MLP 7 -> 64 -> 64 -> C (ReLU), one
// output per tile config (native configs first, then the emulated path's),
// trained on the autotuner's timings to predict ln(time / best time) of every
// config for an unseen (M, N, K, path).  The paper tunes its tile size by hand
// per architecture (Sect. 3, Table 4); the model generalises that sweep.
//
// Kernels (all hand-written, FP32, fixed summation order, so results are
// deterministic):
//   features   x = (log2 M, log2 N, log2 K, log2 M/N, log2 N/K, log2 M/K, path),
//              standardised with a per-feature mean and standard deviation;
//   forward    z1 = W1 x + b1, h1 = relu(z1), z2 = W2 h1 + b2, h2 = relu(z2),
//              y = W3 h2 + b3 (one block of 64 threads per sample);
//   backward   masked MSE L = sum m (y - t)^2 / sum m: per-sample deltas, then
//              one thread per parameter summing its gradient over the batch;
//   adam       elementwise Adam with bias correction (Kingma and Ba 2015).
// Parameters are one float array: W1[64][7], b1[64], W2[64][64], b2[64],
// W3[C][64], b3[C].
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "alp_ext.h"
#include "alp_internal.cuh"

namespace alp {

std::vector<alp_config> configs_of(alp_path path);

namespace {

constexpr int kF = 7, kH = 64;

__host__ __device__ constexpr int64_t off_w1() { return 0; }
__host__ __device__ constexpr int64_t off_b1() { return kH * kF; }
__host__ __device__ constexpr int64_t off_w2() { return kH * kF + kH; }
__host__ __device__ constexpr int64_t off_b2() { return kH * kF + kH + kH * kH; }
__host__ __device__ constexpr int64_t off_w3() { return kH * kF + 2 * kH + kH * kH; }
__host__ __device__ inline int64_t off_b3(int C) { return off_w3() + (int64_t)C * kH; }
__host__ __device__ inline int64_t param_count(int C) { return off_b3(C) + C; }

__global__ void features_kernel(int64_t n, const int64_t* __restrict__ M,
                                const int64_t* __restrict__ N, const int64_t* __restrict__ K,
                                const int32_t* __restrict__ path, const float* __restrict__ mean,
                                const float* __restrict__ stdv, float* __restrict__ X) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float lm = log2f((float)M[i]), ln = log2f((float)N[i]), lk = log2f((float)K[i]);
    float f[kF] = {lm, ln, lk, lm - ln, ln - lk, lm - lk, (float)path[i]};
#pragma unroll
    for (int j = 0; j < kF; ++j) {
        float v = f[j];
        if (mean) v = (v - mean[j]) / stdv[j];
        X[i * kF + j] = v;
    }
}

// mean and standard deviation (population; 1 where it would be 0) per feature
__global__ void stats_kernel(int64_t n, const float* __restrict__ X, float* mean, float* stdv) {
    const int j = threadIdx.x;
    if (j >= kF) return;
    double s = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double v = X[i * kF + j];
        s += v;
        s2 += v * v;
    }
    const double mu = n > 0 ? s / n : 0.0;
    double var = n > 0 ? s2 / n - mu * mu : 0.0;
    if (var < 1e-12) var = 1.0;
    mean[j] = (float)mu;
    stdv[j] = (float)sqrt(var);
}

__global__ void __launch_bounds__(kH) forward_kernel(const float* __restrict__ P, int C,
                                                     const float* __restrict__ X, int64_t B,
                                                     float* __restrict__ Y, float* __restrict__ cache) {
    __shared__ float x[kF], h1[kH], h2[kH];
    const int64_t n = blockIdx.x;
    const int t = threadIdx.x;
    if (t < kF) x[t] = X[n * kF + t];
    __syncthreads();
    float z = P[off_b1() + t];
    for (int f = 0; f < kF; ++f) z += P[off_w1() + t * kF + f] * x[f];
    cache[n * 2 * kH + t] = z;
    h1[t] = z > 0.f ? z : 0.f;
    __syncthreads();
    z = P[off_b2() + t];
    for (int j = 0; j < kH; ++j) z += P[off_w2() + t * kH + j] * h1[j];
    cache[n * 2 * kH + kH + t] = z;
    h2[t] = z > 0.f ? z : 0.f;
    __syncthreads();
    for (int c = t; c < C; c += kH) {
        float y = P[off_b3(C) + c];
        for (int j = 0; j < kH; ++j) y += P[off_w3() + (int64_t)c * kH + j] * h2[j];
        Y[n * C + c] = y;
    }
}

// loss = sum m (y - t)^2 / sum m, and that mask count, into out[0], out[1]
__global__ void loss_kernel(int64_t total, const float* __restrict__ Y, const float* __restrict__ T,
                            const float* __restrict__ Mk, float* out) {
    __shared__ double s[256], c[256];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
        const double d = (double)Y[i] - (double)T[i];
        a += Mk[i] * d * d;
        b += Mk[i];
    }
    s[threadIdx.x] = a;
    c[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s[threadIdx.x] += s[threadIdx.x + o];
            c[threadIdx.x] += c[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = (float)(c[0] > 0 ? s[0] / c[0] : 0.0);
        out[1] = (float)c[0];
    }
}

// per-sample deltas: dy = 2 m (y - t) / count, dz2 = (W3^T dy) * [z2 > 0],
// dz1 = (W2^T dz2) * [z1 > 0]
__global__ void __launch_bounds__(kH) delta_kernel(const float* __restrict__ P, int C,
                                                   int64_t B, const float* __restrict__ cache,
                                                   const float* __restrict__ Y,
                                                   const float* __restrict__ T,
                                                   const float* __restrict__ Mk,
                                                   const float* __restrict__ lossc,
                                                   float* __restrict__ dy,
                                                   float* __restrict__ dz) {
    __shared__ float sdz2[kH];
    const int64_t n = blockIdx.x;
    const int t = threadIdx.x;
    const float inv = lossc[1] > 0.f ? 1.0f / lossc[1] : 0.f;
    for (int c = t; c < C; c += kH) {
        const int64_t i = n * C + c;
        dy[i] = 2.0f * Mk[i] * (Y[i] - T[i]) * inv;
    }
    __syncthreads();
    float g = 0.f;
    for (int c = 0; c < C; ++c) g += P[off_w3() + (int64_t)c * kH + t] * dy[n * C + c];
    const float z2 = cache[n * 2 * kH + kH + t];
    const float d2 = z2 > 0.f ? g : 0.f;
    sdz2[t] = d2;
    dz[n * 2 * kH + kH + t] = d2;
    __syncthreads();
    g = 0.f;
    for (int j = 0; j < kH; ++j) g += P[off_w2() + (int64_t)j * kH + t] * sdz2[j];
    const float z1 = cache[n * 2 * kH + t];
    dz[n * 2 * kH + t] = z1 > 0.f ? g : 0.f;
}

// one thread per parameter: its gradient summed over the batch in sample order
__global__ void grad_kernel(const float* __restrict__ X, int C, int64_t B,
                            const float* __restrict__ cache, const float* __restrict__ dy,
                            const float* __restrict__ dz, float* __restrict__ G) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= param_count(C)) return;
    float s = 0.f;
    if (p < off_b1()) {                        // W1[i][f]
        const int i = (int)(p / kF), f = (int)(p % kF);
        for (int64_t n = 0; n < B; ++n) s += dz[n * 2 * kH + i] * X[n * kF + f];
    } else if (p < off_w2()) {                 // b1[i]
        const int i = (int)(p - off_b1());
        for (int64_t n = 0; n < B; ++n) s += dz[n * 2 * kH + i];
    } else if (p < off_b2()) {                 // W2[i][j]: dz2_i * h1_j
        const int64_t q = p - off_w2();
        const int i = (int)(q / kH), j = (int)(q % kH);
        for (int64_t n = 0; n < B; ++n) {
            const float z1 = cache[n * 2 * kH + j];
            s += dz[n * 2 * kH + kH + i] * (z1 > 0.f ? z1 : 0.f);
        }
    } else if (p < off_w3()) {                 // b2[i]
        const int i = (int)(p - off_b2());
        for (int64_t n = 0; n < B; ++n) s += dz[n * 2 * kH + kH + i];
    } else if (p < off_b3(C)) {                // W3[c][j]: dy_c * h2_j
        const int64_t q = p - off_w3();
        const int c = (int)(q / kH), j = (int)(q % kH);
        for (int64_t n = 0; n < B; ++n) {
            const float z2 = cache[n * 2 * kH + kH + j];
            s += dy[n * C + c] * (z2 > 0.f ? z2 : 0.f);
        }
    } else {                                   // b3[c]
        const int c = (int)(p - off_b3(C));
        for (int64_t n = 0; n < B; ++n) s += dy[n * C + c];
    }
    G[p] = s;
}

__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G,
                            float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---- the model consulted by alp_tune(PREDICT) and by cfg == NULL calls ----
struct Model {
    bool loaded = false;
    int C = 0;
    std::vector<float> params;
    float mean[kF], stdv[kF];
    int dev = -1;
    float* d_params = nullptr;
    float* d_scratch = nullptr;   // X (7) + Y (C) + cache (128)
    int64_t* d_shape = nullptr;   // M, N, K, path
};
std::mutex g_mmu;
Model g_model;

}  // namespace

// Arg-min of the model's predicted log-time over the valid configs of `path`.
bool model_predict(int64_t M, int64_t N, int64_t K, alp_path path, alp_config* out,
                   double* pred_tflops) {
    std::lock_guard<std::mutex> lk(g_mmu);
    if (!g_model.loaded || M <= 0 || N <= 0 || K <= 0) return false;
    const std::vector<alp_config> nat = configs_of(ALP_PATH_NATIVE);
    const std::vector<alp_config> emu = configs_of(ALP_PATH_EMUL);
    if (g_model.C != (int)(nat.size() + emu.size())) return false;
    int dev = 0;
    cudaGetDevice(&dev);
    const int C = g_model.C;
    if (g_model.dev != dev || !g_model.d_params) {
        if (g_model.d_params) cudaFree(g_model.d_params);
        if (g_model.d_scratch) cudaFree(g_model.d_scratch);
        if (g_model.d_shape) cudaFree(g_model.d_shape);
        g_model.d_params = g_model.d_scratch = nullptr;
        g_model.d_shape = nullptr;
        // one-time upload of the model to this device
        if (cudaMalloc(&g_model.d_params, param_count(C) * 4) != cudaSuccess ||
            cudaMalloc(&g_model.d_scratch, (kF + C + 2 * kH + 2 * kF) * 4) != cudaSuccess ||
            cudaMalloc(&g_model.d_shape, 4 * 8) != cudaSuccess)
            return false;
        float ms[2 * kF];
        std::memcpy(ms, g_model.mean, sizeof g_model.mean);
        std::memcpy(ms + kF, g_model.stdv, sizeof g_model.stdv);
        // scratch layout: X (7) | Y (C) | cache (128) | mean, std (14)
        if (cudaMemcpy(g_model.d_params, g_model.params.data(), param_count(C) * 4,
                       cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(g_model.d_scratch + kF + C + 2 * kH, ms, sizeof ms,
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return false;
        g_model.dev = dev;
    }
    float* X = g_model.d_scratch;
    float* Y = X + kF;
    float* cache = Y + C;
    float* ms = cache + 2 * kH;
    const int64_t h_shape[4] = {M, N, K, path == ALP_PATH_EMUL ? 1 : 0};
    const int32_t h_path = (int32_t)h_shape[3];
    if (cudaMemcpy(g_model.d_shape, h_shape, sizeof h_shape, cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    if (cudaMemcpy(reinterpret_cast<char*>(g_model.d_shape) + 24, &h_path, 4,
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    features_kernel<<<1, 32>>>(1, g_model.d_shape, g_model.d_shape + 1, g_model.d_shape + 2,
                               reinterpret_cast<int32_t*>(g_model.d_shape + 3), ms, ms + kF, X);
    forward_kernel<<<1, kH>>>(g_model.d_params, C, X, 1, Y, cache);
    std::vector<float> y(C);
    if (cudaMemcpy(y.data(), Y, C * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    const int lo = path == ALP_PATH_NATIVE ? 0 : (int)nat.size();
    const int hi = path == ALP_PATH_NATIVE ? (int)nat.size() : C;
    int best = lo;
    for (int c = lo; c < hi; ++c)
        if (y[c] < y[best]) best = c;
    *out = path == ALP_PATH_NATIVE ? nat[best] : emu[best - lo];
    if (pred_tflops) *pred_tflops = (double)y[best];   // predicted ln(time / best time)
    return true;
}

}  // namespace alp

using namespace alp;

extern "C" {

int64_t alp_mlp_param_count(int C) { return C > 0 ? param_count(C) : -1; }

alp_status alp_mlp_features(int64_t count, const int64_t* dM, const int64_t* dN,
                            const int64_t* dK, const int32_t* dpath, const float* mean,
                            const float* stdv, float* X, void* stream) {
    if (count < 0 || (count > 0 && (!dM || !dN || !dK || !dpath || !X)) || (!mean != !stdv))
        return ALP_ERR_INVALID_ARG;
    if (count == 0) return ALP_OK;
    features_kernel<<<(unsigned)((count + 255) / 256), 256, 0,
                      reinterpret_cast<cudaStream_t>(stream)>>>(count, dM, dN, dK, dpath, mean,
                                                                stdv, X);
    return cuda_status(cudaGetLastError());
}

alp_status alp_mlp_feature_stats(int64_t count, const float* X, float* mean, float* stdv,
                                 void* stream) {
    if (count < 0 || !X || !mean || !stdv) return ALP_ERR_INVALID_ARG;
    stats_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(count, X, mean, stdv);
    return cuda_status(cudaGetLastError());
}

alp_status alp_mlp_forward(const float* params, int C, const float* X, int64_t B, float* Y,
                           float* cache, void* stream) {
    if (C <= 0 || B < 0 || B > 0x7fffffff || !params || (B > 0 && (!X || !Y || !cache)))
        return ALP_ERR_INVALID_ARG;
    if (B == 0) return ALP_OK;
    forward_kernel<<<(unsigned)B, kH, 0, reinterpret_cast<cudaStream_t>(stream)>>>(params, C, X, B,
                                                                                 Y, cache);
    return cuda_status(cudaGetLastError());
}

alp_status alp_mlp_backward(const float* params, int C, const float* X, int64_t B,
                            const float* cache, const float* Y, const float* T, const float* Mask,
                            float* grads, float* work, float* loss_out, void* stream) {
    if (C <= 0 || B <= 0 || B > 0x7fffffff || !params || !X || !cache || !Y || !T || !Mask ||
        !grads || !work || !loss_out)
        return ALP_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float* dy = work;
    float* dz = work + B * C;
    loss_kernel<<<1, 256, 0, st>>>(B * C, Y, T, Mask, loss_out);
    delta_kernel<<<(unsigned)B, kH, 0, st>>>(params, C, B, cache, Y, T, Mask, loss_out, dy, dz);
    const int64_t P = param_count(C);
    grad_kernel<<<(unsigned)((P + 127) / 128), 128, 0, st>>>(X, C, B, cache, dy, dz, grads);
    return cuda_status(cudaGetLastError());
}

alp_status alp_mlp_adam(float* params, const float* grads, float* m, float* v, int64_t n,
                        int step, float lr, float beta1, float beta2, float eps, void* stream) {
    if (n < 0 || step < 1 || !params || !grads || !m || !v) return ALP_ERR_INVALID_ARG;
    if (n == 0) return ALP_OK;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        params, grads, m, v, n, lr, beta1, beta2, eps, c1, c2);
    return cuda_status(cudaGetLastError());
}

alp_status alp_tune_load_model(const float* host_params, int C, const float* host_mean,
                               const float* host_std) {
    if (!host_params || !host_mean || !host_std || C <= 0) return ALP_ERR_INVALID_ARG;
    const int want = (int)(configs_of(ALP_PATH_NATIVE).size() + configs_of(ALP_PATH_EMUL).size());
    if (C != want) return ALP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mmu);
    g_model.params.assign(host_params, host_params + param_count(C));
    std::memcpy(g_model.mean, host_mean, sizeof g_model.mean);
    std::memcpy(g_model.stdv, host_std, sizeof g_model.stdv);
    g_model.C = C;
    g_model.loaded = true;
    g_model.dev = -1;    // re-upload on next use
    return ALP_OK;
}

alp_status alp_tune_unload_model(void) {
    std::lock_guard<std::mutex> lk(g_mmu);
    g_model.loaded = false;
    return ALP_OK;
}

}  // extern "C"
