// Shared declarations of the emulated FP64 GEMM (emul.cu, emul_gemm.cu).
#pragma once

#include <cuda_bf16.h>

#include "alp_internal.cuh"

namespace alp {

// Digits of b bits, b = 7 (ALP_SLICE_BF16) or 8 (ALP_SLICE_BF16_B8): |d_1| <= 2^b,
// |d_p| <= 2^(b-1), all exact in bf16 (integers up to 256).
constexpr int kDigitBits = 7;
constexpr int kMinSlices = 3;
constexpr int kMaxSlices = 8;      // array bound; per digit width see emul_max_slices
constexpr int kEmulBK = 64;        // K elements per pipeline stage (128 bytes of bf16)
// Most slices per digit width: the split's 62-bit fixed point stays exact
// while (s - 1) * b + 2 <= 62 - b.
inline int emul_max_slices(int b) { return b == 8 ? 7 : 8; }
// FP32 results: s b <= 32 keeps the exact sum in 64 bits.
inline int emul_max_slices_f32(int b) { return 32 / b; }
// Largest K per call: the int32 group sums |S^t| <= K * 2^(2b-2) * (t + 1),
// t <= s + 1, stay below 2^31 (b = 7: K <= 32768; b = 8: K <= 14336).
inline int64_t emul_max_k(int b) { return b == 8 ? 14336 : 32768; }
constexpr int64_t kEmulMaxK = 32768;
inline bool emul_digit_bits_ok(int b) { return b == 7 || b == 8; }

// The scheme of a slice kind: b bits per digit, whether the last group t =
// s+1 is trimmed to its pairs with a leading digit, (1, s) and (s, 1), or
// the modular scheme (residues modulo s pairwise coprime moduli; b = 8 is
// its residue width for the chunk bounds).
struct EmulScheme {
    int b;
    bool trim;
    bool crt;
};
inline bool emul_scheme_of(int kind, EmulScheme* sc) {
    switch (kind) {
        case ALP_SLICE_BF16: *sc = {7, false, false}; return true;
        case ALP_SLICE_BF16_B8: *sc = {8, false, false}; return true;
        case ALP_SLICE_BF16_B8_TRIM: *sc = {8, true, false}; return true;
        case ALP_SLICE_BF16_CRT: *sc = {8, false, true}; return true;
        default: return false;
    }
}

// The modular scheme (emul_crt.cu): 4..16 moduli; k = crt_bits(K, n) bits per
// scaled operand (0 when no k >= 1 fits).
constexpr int kCrtMinModuli = 4;
constexpr int kCrtMaxModuli = 16;
// Largest K of the modular scheme: 1023 k-blocks of 64 (the job encoding),
// where the exact sums |Q_l| <= K 2^14 < 2^30 stay within the residue
// reduction's range.
constexpr int64_t kCrtMaxK = 1023 * 64;
int crt_bits(int64_t K, int n);
// y_l = (Mn / m_l)^-1 mod m_l for the first n moduli (host).
uint32_t crt_weight(int n, int l);
template <typename T>
alp_status emul_split_crt(int64_t R, int64_t K, const T* X, int64_t ldx, int trans,
                          const int32_t* exps, int n, __nv_bfloat16* out, int64_t kpad, int k,
                          cudaStream_t st);
// Rows of a row-major R x K double matrix: the exponent scan and the residue
// split in one pass per row (exps written; out 8-byte aligned, kpad % 4 == 0).
alp_status emul_scan_split_crt(int64_t R, int64_t K, const double* X, int64_t ldx,
                               int32_t* exps, int n, __nv_bfloat16* out, int64_t kpad, int k,
                               cudaStream_t st);
alp_status launch_recombine_crt(int n, int k, dim3 grid, cudaStream_t st, const uint8_t* R,
                                int64_t rplane, int64_t ldr, const int32_t* e, const int32_t* f,
                                int64_t M, int64_t N, double alpha, double beta, double* C,
                                int64_t ldc);
// Slice counts a GEMM call accepts: 3..emul_max_slices(b) digits for FP64,
// 2..32/b for FP32, kCrtMinModuli..kCrtMaxModuli moduli for the modular scheme.
inline bool emul_slices_ok(const EmulScheme& sc, int s, bool f32) {
    if (sc.crt) return !f32 && s >= kCrtMinModuli && s <= kCrtMaxModuli;
    return f32 ? (s >= 2 && s <= emul_max_slices_f32(sc.b))
               : (s >= kMinSlices && s <= emul_max_slices(sc.b));
}
// Largest K of one call.
inline int64_t emul_scheme_max_k(const EmulScheme& sc) {
    return sc.crt ? kCrtMaxK : emul_max_k(sc.b);
}
// Whether digit pair (p, q) of group t = p + q is multiplied.
__host__ __device__ inline bool emul_pair_kept(int p, int q, int s, bool trim) {
    return p + q <= s + 1 && (!trim || p + q <= s || p == 1 || q == 1);
}

struct EmulLayout {
    int64_t kpad;    // K rounded up to kEmulBK (digit rows, zero filled)
    int64_t ldg;     // row stride of the int32 group sums (N rounded up to 256)
    size_t off_da, off_db, off_g, off_e, off_f, bytes;
    size_t off_sched, sched_bytes;   // the modular scheme's fused schedule (gbytes 1)
};

// gbytes: bytes per element of G (4: int32 group sums; 1: the modular
// scheme's residues).
EmulLayout emul_layout(int64_t M, int64_t N, int64_t K, int s, int gbytes = 4);

// Block arrangement of the slice-product kernel: one block per 128 x 256
// tile, or a CTA pair whose MMAs span both SMs (tcgen05 .cta_group::2,
// 256 x 256 per pair).
enum EmulArrangement { kEmulSingle = 1, kEmulPair = 3 };

// S^t for t = 2..s+1 into G[(t-2)][M][ldg] (int32), from the digit slices
// da[s][M][kpad] and db[s][N][kpad] (bf16, K-major); with crt, s moduli and
// the residue slices instead, and G holds s byte planes [l][M][ldg] of
// (Q_l y_l) mod m_l.  group_m: tile-rows per raster group (0 = default, the
// tunable of the emulated path).  cluster: the EmulArrangement (0 = default,
// emul_cluster()).
alp_status emul_slice_gemm(int64_t M, int64_t N, int64_t K, int s, const __nv_bfloat16* da,
                           const __nv_bfloat16* db, int64_t kpad, int32_t* G, int64_t ldg,
                           cudaStream_t stream, int group_m = 0, int cluster = 0,
                           int digit_bits = kDigitBits, bool trim = false, bool crt = false);

// Grid of the reconstruction kernels: 512 columns per block, rows strided.
dim3 recombine_grid(int64_t M, int64_t N);

// The modular scheme's products and reconstruction: C = alpha RN(P 2^(e_i +
// f_j - 2k)) (+ beta C) from the n residue slices, with G (n byte planes, row
// stride ldg bytes, a multiple of 256) as the residue workspace.  With the
// CTA-pair arrangement one persistent launch reconstructs each tile while the
// next one's products run (emul_gemm.cu), then the tail tiles; otherwise (or
// with ALP_EMUL_CRT_FUSE=0) the product stage and the reconstruction kernel.
// sched: the fused launch's schedule (emul_crt_sched_bytes(M, N) bytes of
// device memory, 4-byte aligned; without it the two launches run).  fuse: 1
// fuse, 0 do not, -1 as ALP_EMUL_CRT_FUSE says.
alp_status emul_crt_products_recombine(int64_t M, int64_t N, int64_t K, int n,
                                       const __nv_bfloat16* da, const __nv_bfloat16* db,
                                       int64_t kpad, uint8_t* G, int64_t ldg, const int32_t* e,
                                       const int32_t* f, int k, double alpha, double beta,
                                       double* C, int64_t ldc, int* sched, size_t sched_bytes,
                                       cudaStream_t stream, int group_m = 0, int cluster = 0,
                                       int fuse = -1);
size_t emul_crt_sched_bytes(int64_t M, int64_t N);

// Tail split of the slice-product launch (see emul_gemm.cu): whole tiles for
// blocks [0, n_full), then each remaining tile cut into `pieces` blocks by
// group ranges t_lo[i]..t_hi[i].
struct TailSplit {
    int n_full, pieces;
    int t_lo[8], t_hi[8];
};
TailSplit tail_split(int tiles, int s, int sms, bool trim = false, bool crt = false);

// Configs of the emulated path: alp_config{128, 256, 64, 1, 0, group_m} (one
// block per tile) or {256, 256, 64, 2, 0, group_m} (CTA pairs sharing each
// MMA), and group_m in {1, 2, 4, 8, 16, 32} (tile-rows per raster group).
inline bool emul_config_valid(const alp_config& c) {
    const bool group = c.stages == 1 || c.stages == 2 || c.stages == 4 || c.stages == 8 ||
                       c.stages == 16 || c.stages == 32;
    const bool single = c.bm == 128 && c.tm == 1;
    const bool pair = c.bm == 256 && c.tm == 2;
    return (single || pair) && c.bn == 256 && c.bk == 64 && c.tn == 0 && group;
}
// The EmulArrangement of a valid config.
inline int emul_arrangement_of(const alp_config& c) {
    return c.bm == 256 ? kEmulPair : kEmulSingle;
}

}  // namespace alp
