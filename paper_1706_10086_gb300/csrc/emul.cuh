// Shared declarations of the emulated FP64 GEMM (emul.cu, emul_gemm.cu).
#pragma once

#include <cuda_bf16.h>

#include "alp_internal.cuh"

namespace alp {

constexpr int kDigitBits = 7;      // b: bits per digit; digits |d| <= 128 are exact in bf16
constexpr int kMinSlices = 3;
constexpr int kMaxSlices = 8;      // s * b <= 56 keeps the split's fixed point exact
constexpr int kEmulBK = 64;        // K elements per pipeline stage (128 bytes of bf16)
// Largest K per call: the int32 group sums |S^t| <= K * 2^12 * (t + 1) (t <= 9)
// stay below 2^31 for K <= 32768.
constexpr int64_t kEmulMaxK = 32768;

struct EmulLayout {
    int64_t kpad;    // K rounded up to kEmulBK (digit rows, zero filled)
    int64_t ldg;     // row stride of the int32 group sums (N rounded up to 256)
    size_t off_da, off_db, off_g, off_e, off_f, bytes;
};

EmulLayout emul_layout(int64_t M, int64_t N, int64_t K, int s);

// S^t for t = 2..s+1 into G[(t-2)][M][ldg] (int32), from the digit slices
// da[s][M][kpad] and db[s][N][kpad] (bf16, K-major).  group_m: tile-rows per
// raster group (0 = default, the tunable of the emulated path).
// cluster: blocks per cluster sharing B tiles (1 or 2; 0 = default 1).
alp_status emul_slice_gemm(int64_t M, int64_t N, int64_t K, int s, const __nv_bfloat16* da,
                           const __nv_bfloat16* db, int64_t kpad, int32_t* G, int64_t ldg,
                           cudaStream_t stream, int group_m = 0, int cluster = 0);

// Configs of the emulated path: alp_config{128, 256, 64, cluster, 0, group_m}
// with cluster in {1, 2} (blocks sharing each B tile) and group_m in
// {1, 2, 4, 8, 16, 32} (tile-rows per raster group); the tile is fixed.
inline bool emul_config_valid(const alp_config& c) {
    return c.bm == 128 && c.bn == 256 && c.bk == 64 && (c.tm == 1 || c.tm == 2) && c.tn == 0 &&
           (c.stages == 1 || c.stages == 2 || c.stages == 4 || c.stages == 8 || c.stages == 16 ||
            c.stages == 32);
}

}  // namespace alp
