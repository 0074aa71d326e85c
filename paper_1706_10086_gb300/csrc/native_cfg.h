// Tile-configuration rules of the native FP64 kernel.  Host and device code of
// the library both include this file, so the validity filter and the kernel
// instantiations agree by construction.
//
// The paper tunes one tile size T per architecture (Sect. 2.1, Listing 1,
// Table 4) with 16x16 threads per block on GPUs.  Here a thread block owns a
// bm x bn tile of C (one C tile per block, Sect. 2.1), steps through K in
// chunks of bk, and each thread owns a tm x tn register tile of C (the element
// layer).  A warp's 32 threads form (8*tm) x (4*tn) of C through m16n8k4 FP64
// MMA fragments (each fragment gives a thread a 2 x 2 block).
#pragma once

#include <stdint.h>

namespace alp {

constexpr int kSmemLimit = 232448;      // 227 KiB opt-in shared memory per block (sm_100+)
constexpr int kSmemReserve = 1024;      // barriers and alignment slack
constexpr int kMaxStages = 4;

// Thread cap of one block of a (tm, tn) instantiation.  Each instantiation is
// compiled with __launch_bounds__(max_threads(tm, tn), 1), so ptxas keeps a
// thread within 65536 / (4 * ceil(warps / 4) * 32) registers: enough for the
// 2*tm*tn registers of the FP64 accumulators plus fragments and addressing
// without spilling (checked with -Xptxas -v).
constexpr int max_threads(int tm, int tn) {
    return (tm == 2 && tn == 2) ? 1024 : (tm == 2 && tn == 4) ? 1024
         : (tm == 2 && tn == 8) ? 768  : (tm == 4 && tn == 2) ? 896
         : (tm == 4 && tn == 4) ? 768  : (tm == 4 && tn == 8) ? 512
         : (tm == 8 && tn == 2) ? 768  : (tm == 8 && tn == 4) ? 512
         : (tm == 8 && tn == 8) ? 384  : 256;
}

inline bool in_set3(int v, int a, int b, int c) { return v == a || v == b || v == c; }

// Threads of one block of the TMA kernel: one producer warp plus the warps
// that compute (bm/(8tm)) x (bn/(4tn)) warp tiles.
inline int native_compute_warps(int bm, int bn, int tm, int tn) {
    return (bm / (8 * tm)) * (bn / (4 * tn));
}
inline int native_threads(int bm, int bn, int tm, int tn) {
    return 32 * (1 + native_compute_warps(bm, bn, tm, tn));
}
inline int64_t native_stage_bytes(int bm, int bn, int bk) {
    return (int64_t)(bm + bn) * bk * 8;
}
// Stages used for a config: the requested count, or as many as fit (<= 4).
inline int native_stages(int bm, int bn, int bk, int requested) {
    int64_t sb = native_stage_bytes(bm, bn, bk);
    int fit = (int)((kSmemLimit - kSmemReserve) / sb);
    if (fit > kMaxStages) fit = kMaxStages;
    if (requested > 0) return requested <= fit ? requested : 0;
    return fit;
}
inline int64_t native_smem_bytes(int bm, int bn, int bk, int stages) {
    return native_stage_bytes(bm, bn, bk) * stages + kSmemReserve;
}

// Static validity of a native config (no GPU needed).
inline bool native_config_valid(int bm, int bn, int bk, int tm, int tn, int stages) {
    if (!in_set3(bm, 64, 128, 256) || !in_set3(bn, 64, 128, 256)) return false;
    if (!in_set3(bk, 16, 32, 64)) return false;
    if (!in_set3(tm, 2, 4, 8) || !in_set3(tn, 2, 4, 8)) return false;
    if (bm % (8 * tm) || bn % (4 * tn)) return false;
    if (native_threads(bm, bn, tm, tn) > max_threads(tm, tn)) return false;
    if (stages < 0 || stages > kMaxStages) return false;
    int s = native_stages(bm, bn, bk, stages);
    return s >= 2;
}

}  // namespace alp
