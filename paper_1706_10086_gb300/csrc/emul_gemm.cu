// Slice products of the emulated FP64 GEMM on tcgen05 tensor cores.
//
// Arrangements (emul_arrangement_of): by default a CTA pair (2-block cluster)
// per 256 x 256 tile of C, its tcgen05 MMAs (.cta_group::2, M = 256) spanning
// both SMs; otherwise one block per 128 x 256 tile.  In the last, partial wave
// each tile is cut into up to 8 blocks (or pairs) by ranges of groups t
// (tail_split below) so that the wave ends sooner.  Per block:
//
//   warp 0      TMA producer: 128x64 A and 256x64 (pair: 128x64) B tiles
//               (128-byte swizzle) into a shared-memory ring of stages
//               ("full"/"empty" mbarriers);
//   warp 1      allocates 512 TMEM columns (two f32 accumulators of 256
//               columns) and issues tcgen05.mma kind::f16 (K = 16) from one
//               thread, committing each stage back to the producer and each
//               finished chunk to the epilogue;
//   warps 2-9   drain a finished chunk from TMEM (tcgen05.ld) while the other
//               accumulator fills, and add it exactly into int32 registers
//               (the CTA-pair kernels: warps 4-11 of 16, with more registers
//               each; kPairThreads).
//
// Jobs (build_jobs): the digit schemes multiply the digit pairs (p, q) of
// each group t = p + q <= s + 1 (groups ascending, p ascending); the modular
// scheme multiplies residue slice l of A by residue slice l of B, one group
// per modulus.  Each job is one K chunk of one product.
//
// Exactness: digits satisfy |d_1| <= 2^b, |d_p| <= 2^(b-1) (p >= 2), so a
// chunk of 2^(24-2b) (pair 1,1), 2^(25-2b) (one first digit) or 2^(26-2b) (no
// first digit) products -- 1024 / 2048 / 4096 for b = 7, 256 / 512 / 1024 for
// b = 8 -- has |partial sum| <= 2^24; residues satisfy |r| <= 128, so chunks
// of 1024 do.  Every value the f32 accumulator takes is then an integer f32
// holds exactly, so no MMA rounds.  The drain converts each chunk's integer
// exactly (cvt) and adds it into a 32-bit running sum, the exact group sum
// (|S^t| < 2^31, |Q_l| <= K 2^14 for the K limits).  At the end of a group
// the block writes S^t to G[t-2] (int32), or, for the modular scheme, the byte
// (Q_l y_l) mod m_l to plane l-1 of G.
#include <cstdlib>

#include "crt.cuh"
#include "crt_rec.cuh"
#include "emul.cuh"
#include "tc.cuh"

namespace alp {

alp_status make_tmap_3d_bf16(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1,
                             uint64_t d2, uint32_t box0, uint32_t box1);

// Block arrangement when the config does not say (env ALP_EMUL_CLUSTER: 1 =
// one block per tile, 3 = CTA pairs sharing each MMA; default 3, the fastest
// at 8192^3 on GB300).
static int emul_cluster() {
    static int c = 0;
    if (c == 0) {
        c = kEmulPair;
        if (const char* s = std::getenv("ALP_EMUL_CLUSTER")) {
            const int v = std::atoi(s);
            if (v == kEmulSingle || v == kEmulPair) c = v;
        }
    }
    return c;
}

// Tile-rows per raster group (env ALP_EMUL_GROUP_M overrides; default the
// fastest at 8192^3 on GB300: 16 for CTA pairs, 8 otherwise).
static int emul_group_m(bool pair) {
    static int g = -1;
    if (g < 0) {
        g = 0;
        if (const char* s = std::getenv("ALP_EMUL_GROUP_M")) {
            const int v = std::atoi(s);
            if (v >= 1 && v <= 4096) g = v;
        }
    }
    return g > 0 ? g : pair ? 16 : 8;
}

// Whether the last partial wave is split (env ALP_EMUL_TAIL_SPLIT=0 turns it
// off; default on).
static bool emul_tail_split_on() {
    static int on = -1;
    if (on < 0) {
        const char* s = std::getenv("ALP_EMUL_TAIL_SPLIT");
        on = (s && std::atoi(s) == 0) ? 0 : 1;
    }
    return on == 1;
}

// Whether alp_gemm_f64_emul's modular scheme reconstructs C inside the
// product kernel (env ALP_EMUL_CRT_FUSE=0 turns it off: products, then the
// reconstruction kernel; default on).  Only the CTA-pair arrangement fuses.
static bool emul_crt_fuse_on() {
    static int on = -1;
    if (on < 0) {
        const char* s = std::getenv("ALP_EMUL_CRT_FUSE");
        on = (s && std::atoi(s) == 0) ? 0 : 1;
    }
    return on == 1;
}

namespace {

constexpr int kTM = 128, kTN = 256, kTK = kEmulBK;
constexpr int kStages = 4;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kATile = kTM * kTK * 2;
constexpr uint32_t kBTile = kTN * kTK * 2;
constexpr uint32_t kStageBytes = kATile + kBTile;
constexpr uint32_t kTmemCols = 2 * kTN;
constexpr int kMaxJobs = 1024;   // >= jobs of one tile: s = 8, b = 7, K = 32768: 424;
                                 // s = 7, b = 8, K = 14336: 602
constexpr int kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/ + 4 * kMaxJobs;

struct EmulGemmParams {
    int64_t M, N, K;
    int s, digit_bits, trim, crt;
    int32_t* G;
    int64_t ldg, gplane;
    int tiles_m, tiles_n, group_m;
    // tail split: blocks [0, n_full) take whole tiles; tiles n_full.. (the last,
    // partial wave) are cut into `pieces` blocks each, piece i taking the
    // groups t_lo..t_hi packed in byte i of t_ranges ((t_lo - 2) | (t_hi - 2) << 4,
    // so that t up to 17, the last group of 16 moduli, fits).
    // Groups write disjoint planes of G.
    int n_full, pieces;
    uint64_t t_ranges;
    uint64_t timeout_ns;
    int* err;
    // test hook: block 0's producer arms pipeline stage inject_skip_it (its
    // running stage count) without issuing the copies (-1: off)
    int64_t inject_skip_it;
    // modular scheme: y_l = (Mn / m_l)^-1 mod m_l, the weight of residue l
    uint8_t crt_y[kCrtMaxModuli];
};

// K chunk of pair (p, q): the largest multiple of 64 with |partial sums| <= 2^24,
// from the product bounds 2^(2b) (p = q = 1), 2^(2b-1) (one first digit),
// 2^(2b-2) (none): 1024 / 2048 / 4096 for b = 7, 256 / 512 / 1024 for b = 8.
__host__ __device__ __forceinline__ int chunk_of(int p, int q, int b) {
    const int e = (p == 1 && q == 1) ? 2 * b : (p == 1 || q == 1) ? 2 * b - 1 : 2 * b - 2;
    return 1 << (24 - e);
}

// The fixed job order of one tile (or of one piece of it, groups t_lo..t_hi):
// groups t ascending, pairs p ascending (q = t - p), K chunks ascending.  One
// 32-bit word per job: first k-block (bits 0..9), end k-block (10..19), p-1
// (20..23), q-1 (24..27), last chunk of its group (28).  Thread 0 writes the
// table into shared memory; every role walks it.  Returns the number of jobs.
__device__ int build_jobs(int s, int K, int b, bool trim, bool crt, int t_lo, int t_hi,
                          uint32_t* jobs) {
    int n = 0;
    const int kblocks = (K + kTK - 1) / kTK;
    for (int t = t_lo; t <= t_hi; ++t) {
        if (crt) {
            // modular scheme: group t is modulus l = t - 1, the pair (l, l);
            // residues |r| <= 128, so chunks of 1024 keep partial sums <= 2^24
            const int l = t - 1, cb = 1024 / kTK;
            for (int kb = 0; kb < kblocks; kb += cb) {
                const int ke = (kb + cb < kblocks) ? kb + cb : kblocks;
                const uint32_t last = ke == kblocks ? 1u : 0u;
                jobs[n++] = (uint32_t)kb | ((uint32_t)ke << 10) | ((uint32_t)(l - 1) << 20) |
                            ((uint32_t)(l - 1) << 24) | (last << 28);
            }
            continue;
        }
        const int plo = (t - s > 1) ? t - s : 1;
        int phi = (s < t - 1) ? s : t - 1;
        while (phi > plo && !emul_pair_kept(phi, t - phi, s, trim)) --phi;   // last kept pair
        for (int p = plo; p <= phi; ++p) {
            const int q = t - p;
            if (!emul_pair_kept(p, q, s, trim)) continue;
            const int cb = chunk_of(p, q, b) / kTK;
            for (int kb = 0; kb < kblocks; kb += cb) {
                const int ke = (kb + cb < kblocks) ? kb + cb : kblocks;
                const uint32_t last = (ke == kblocks && p == phi) ? 1u : 0u;
                jobs[n++] = (uint32_t)kb | ((uint32_t)ke << 10) | ((uint32_t)(p - 1) << 20) |
                            ((uint32_t)(q - 1) << 24) | (last << 28);
            }
        }
    }
    return n;
}
__device__ __forceinline__ int job_kb(uint32_t j) { return (int)(j & 1023u); }
__device__ __forceinline__ int job_ke(uint32_t j) { return (int)((j >> 10) & 1023u); }
__device__ __forceinline__ int job_p(uint32_t j) { return (int)((j >> 20) & 15u) + 1; }
__device__ __forceinline__ int job_q(uint32_t j) { return (int)((j >> 24) & 15u) + 1; }
__device__ __forceinline__ bool job_last(uint32_t j) { return (j >> 28) & 1u; }

// g[0..3] = a[0..3] (if do_store), then a[0..3] = 0.
__device__ __forceinline__ void store4_and_zero(int32_t* g, uint32_t do_store, uint32_t& a0,
                                                uint32_t& a1, uint32_t& a2, uint32_t& a3) {
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.u32 p, %5, 0;\n"
        " @p st.global.v4.b32 [%4], {%0, %1, %2, %3};\n"
        " mov.b32 %0, 0;\n mov.b32 %1, 0;\n mov.b32 %2, 0;\n mov.b32 %3, 0;\n"
        "}\n"
        : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3)
        : "l"(g), "r"(do_store)
        : "memory");
}

// Hands accumulator b back to the MMA thread after this warp's drain of job
// `job`: an arrive on acce[b] of this block, or, in block 1 of a CTA pair
// (acce_remote = the shared::cluster address of block 0's acce), an arrive on
// the local agg[b]; warp 2 waits for all kEpiWarps of them and then forwards
// them to block 0 as one remote arrival of that count (remote arrivals from
// one SM take their turns, so eight per chunk lengthen the hand-back).  A wait
// that gives up leaves the hand-back undone; the launch is aborting.
__device__ __forceinline__ void hand_back(uint64_t* acce, uint32_t acce_remote, uint64_t* agg,
                                          uint32_t b, int job, int warp, uint64_t tmo,
                                          volatile int* abort_flag, int* err) {
    if (!acce_remote) {
        mbar_arrive(&acce[b]);
        return;
    }
    mbar_arrive(&agg[b]);
    if (warp == 2 && mbar_wait_bounded(&agg[b], (job >> 1) & 1, tmo, abort_flag, err))
        mbar_arrive_cluster(acce_remote + b * 8, kEpiWarps);
}

// Epilogue warps (2..9): for each finished chunk, drain this warp's 32 TMEM
// lanes x 128 columns of accumulator b into exact int32 sums, hand the
// accumulator back (hand_back), and at the end of a group store S^t to
// G[t-2].
__device__ __forceinline__ void epilogue_role(const EmulGemmParams& prm, const uint32_t* jobs,
                                              int njobs, uint32_t tmem_base, uint64_t* accf,
                                              uint64_t* acce, uint32_t acce_remote, uint64_t* agg,
                                              int m0, int n0, int warp, int lane, uint64_t tmo,
                                              volatile int* abort_flag, int ew) {
    // ew: this warp's index among the eight epilogue warps (the first one
    // forwards block 1's hand-backs); warp: its index in the block, whose
    // value modulo 4 fixes the TMEM lanes it may access
    const int quarter = warp & 3;
    const int half = ew >> 2;              // columns [128*half, 128*half + 128)
    const int row = quarter * 32 + lane;
    const int gm = m0 + row;
    uint32_t acc[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) acc[i] = 0;
    int t_group = 2;
    for (int job = 0; job < njobs; ++job) {
        const uint32_t b = job & 1;
        if (!mbar_wait_bounded(&accf[b], (job >> 1) & 1, tmo, abort_flag, prm.err)) break;
        tc_fence_after();
        const uint32_t taddr =
            tmem_base + ((uint32_t)(quarter * 32) << 16) + b * kTN + half * 128;
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_drain32_cvt(taddr + c * 32, &acc[c * 32]);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) hand_back(acce, acce_remote, agg, b, job, ew + 2, tmo, abort_flag, prm.err);
        const uint32_t jd = jobs[job];
        if (job_last(jd) && prm.crt) {
            // modular scheme: plane l of modulus m_l receives x = (Q y_l) mod
            // m_l = (P y_l) mod m_l, one byte per column (rows padded as below)
            const int l = job_p(jd) - 1;
            const uint32_t m = crt_modulus(l), magic = crt_magic(m), y = prm.crt_y[l];
            uint8_t* g = reinterpret_cast<uint8_t*>(prm.G) + (int64_t)l * prm.gplane +
                         (int64_t)gm * prm.ldg + n0 + half * 128;
            const uint32_t do_store = gm < prm.M ? 1u : 0u;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = 16 * i + 4 * q;
                    w[q] = crt_mod(crt_residue((int32_t)acc[c], m, magic) * y, m, magic) |
                           crt_mod(crt_residue((int32_t)acc[c + 1], m, magic) * y, m, magic) << 8 |
                           crt_mod(crt_residue((int32_t)acc[c + 2], m, magic) * y, m, magic) << 16 |
                           crt_mod(crt_residue((int32_t)acc[c + 3], m, magic) * y, m, magic) << 24;
                }
                store4_and_zero(reinterpret_cast<int32_t*>(g + 16 * i), do_store, w[0], w[1],
                                w[2], w[3]);
            }
#pragma unroll
            for (int i = 0; i < 128; ++i) acc[i] = 0;
        } else if (job_last(jd)) {
            // plane of G: t - 2 for the digit pair (p, q), t = p + q
            t_group = job_p(jd) + job_q(jd);
            // G rows are padded to whole 256-column tiles, so the strip is in
            // bounds; rows past M are not stored.  Each asm block stores acc
            // and zeroes it in place.
            int32_t* g = prm.G + (int64_t)(t_group - 2) * prm.gplane + (int64_t)gm * prm.ldg +
                         n0 + half * 128;
            const uint32_t do_store = gm < prm.M ? 1u : 0u;
#pragma unroll
            for (int i = 0; i < 32; ++i)
                store4_and_zero(g + 4 * i, do_store, acc[4 * i], acc[4 * i + 1], acc[4 * i + 2],
                                acc[4 * i + 3]);
        }
    }
}

// One block per 128 x 256 tile.
__global__ void __launch_bounds__(kThreads, 1)
    emul_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB, EmulGemmParams prm) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw_u32 = smem_u32(smem_raw);
    unsigned char* smem = smem_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
    unsigned char* tiles = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* accf = empty + kStages;
    uint64_t* acce = accf + 2;
    uint64_t* done = acce + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* njobs_slot = const_cast<int*>(reinterpret_cast<volatile int*>(abort_flag + 1));
    uint32_t* jobs = reinterpret_cast<uint32_t*>(smem + kStages * kStageBytes + 256);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], kEpiWarps);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        int t_lo = 2, t_hi = prm.s + 1;
        if ((int)blockIdx.x >= prm.n_full) {
            const int pc = ((int)blockIdx.x - prm.n_full) % prm.pieces;
            const uint32_t r = (uint32_t)(prm.t_ranges >> (8 * pc)) & 0xffu;
            t_lo = (int)(r & 15u) + 2;
            t_hi = (int)(r >> 4) + 2;
        }
        *njobs_slot = build_jobs(prm.s, (int)prm.K, prm.digit_bits, prm.trim != 0, prm.crt != 0,
                                 t_lo, t_hi, jobs);
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int njobs = *njobs_slot;

    // grouped raster: blocks run down group_m tile-rows before moving one
    // tile-column right, so a wave of blocks shares a compact set of A and B
    // digit panels in L2
    int m0, n0;
    {
        const int gm = prm.group_m > 0 ? prm.group_m : 1;
        const int pid = (int)blockIdx.x < prm.n_full
                            ? (int)blockIdx.x
                            : prm.n_full + ((int)blockIdx.x - prm.n_full) / prm.pieces;
        const int in_group = gm * prm.tiles_n;
        const int first_m = (pid / in_group) * gm;
        const int gsz = min(prm.tiles_m - first_m, gm);
        const int local = pid % in_group;
        m0 = (first_m + local % gsz) * kTM;
        n0 = (local / gsz) * kTN;
    }
    const uint64_t tmo = prm.timeout_ns;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
            uint32_t it = 0;
            int64_t skipped = -1;
            bool ok = true;
            for (int j = 0; j < njobs && ok; ++j) {
                const uint32_t jd = jobs[j];
                for (int kb = job_kb(jd); kb < job_ke(jd); ++kb, ++it) {
                    const uint32_t st = it % kStages, round = it / kStages;
                    if (it >= (uint32_t)kStages &&
                        !mbar_wait_bounded(&empty[st], (round - 1) & 1, tmo, abort_flag, prm.err)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], kStageBytes);
                    if ((int64_t)it == prm.inject_skip_it && blockIdx.x == 0) {
                        skipped = it;   // fault injection: the stage never fills
                        continue;
                    }
                    unsigned char* a = tiles + st * kStageBytes;
                    tma_load_3d(a, &tmA, &full[st], kb * kTK, m0, job_p(jd) - 1);
                    tma_load_3d(a + kATile, &tmB, &full[st], kb * kTK, n0, job_q(jd) - 1);
                }
            }
            // every copy issued must land before the block may exit
            for (uint32_t j = it > (uint32_t)kStages ? it - kStages : 0; j < it; ++j)
                if ((int64_t)j != skipped)
                    mbar_wait_bounded(&full[j % kStages], (j / kStages) & 1, tmo, nullptr,
                                      prm.err, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = idesc_bf16_f32(kTM, kTN);
            uint32_t it = 0;
            bool ok = true;
            for (int job = 0; job < njobs && ok; ++job) {
                const uint32_t jd = jobs[job];
                const uint32_t b = job & 1;
                if (job >= 2 &&
                    !mbar_wait_bounded(&acce[b], ((job >> 1) - 1) & 1, tmo, abort_flag, prm.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + b * kTN;
                uint32_t accumulate = 0;
                for (int kb = job_kb(jd); kb < job_ke(jd); ++kb, ++it) {
                    const uint32_t st = it % kStages, round = it / kStages;
                    if (!mbar_wait_bounded(&full[st], round & 1, tmo, abort_flag, prm.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(tiles + st * kStageBytes);
                    const uint64_t adesc = sw128_kmajor_desc(a_addr);
                    const uint64_t bdesc = sw128_kmajor_desc(a_addr + kATile);
#pragma unroll
                    for (int kk = 0; kk < kTK / 16; ++kk) {
                        // +32 bytes along K inside the 128-byte swizzled row
                        umma_bf16(d_tmem, adesc + 2 * kk, bdesc + 2 * kk, idesc, accumulate);
                        accumulate = 1;
                    }
                    umma_commit(&empty[st]);
                }
                if (!ok) break;
                umma_commit(&accf[b]);
            }
            // all MMAs must have completed before TMEM and shared memory go away
            umma_commit(done);
            mbar_wait_bounded(done, 0, tmo, nullptr, prm.err, false);
        }
    } else {
        epilogue_role(prm, jobs, njobs, tmem_base, accf, &acce[0], 0u, nullptr, m0, n0, warp,
                      lane, tmo, abort_flag, warp - 2);
    }
    tc_fence_before();
    __syncwarp();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

// CTA-pair variant (tcgen05 .cta_group::2): a cluster of two blocks computes
// a 256 x 256 tile with M = 256, N = 256 MMAs issued by one thread of block 0.
// Block r holds rows [m0 + 128 r, +128) of A and rows [n0 + 128 r, +128) of
// the K-major B per stage (16 + 16 KB, 6 stages), and its TMEM receives rows
// m0 + 128 r.. of the tile, so each SM stages half the B bytes of the
// one-block kernel per MMA.  Both blocks' copies complete on block 0's "full"
// barriers (its producer expects the bytes of both); the MMA thread releases
// stages and chunks in both blocks by multicast commits; block 1's epilogue
// hands accumulators back on block 0's "acce" barriers.
constexpr int kPairStages = 6;
// Sixteen warps: 0 the TMA producer, 1 the MMA issuer, 4-11 the epilogue;
// the epilogue's warpgroups take 176 registers per thread from the others'
// (setmaxnreg: 2 x 128 x 176 + 2 x 128 x 80 = 65536, the launch's 512 x 128),
// so that its 128 running sums per thread fit without spilling.
constexpr int kPairThreads = 512;
constexpr int kPairEpiRegs = 176, kPairLowRegs = 80;
static_assert(2 * 128 * kPairEpiRegs + 2 * 128 * kPairLowRegs == kPairThreads * 128,
              "register split of the CTA-pair kernel");
// Limit of the pair producer's final waits once the launch has aborted (2 ms).
constexpr uint64_t kDrainNs = 2000000ull;
constexpr uint32_t kPairBTile = kBTile / 2;
constexpr uint32_t kPairStageBytes = kATile + kPairBTile;
constexpr int kPairSmemBytes = kPairStages * kPairStageBytes + 1024 /*align*/ + 256 /*barriers*/ +
                               4 * kMaxJobs;

constexpr int kFusedSmemBytes = kPairStages * kPairStageBytes + 1024 /*align*/ + 256 /*barriers*/;

// Grouped raster in units of 256-row tile pairs: the origin of pair tile pid
// (m0 = the first of the 128 rows block `rank` holds, n0 = the first column).
__device__ __forceinline__ void pair_tile_origin(const EmulGemmParams& prm, int pid, uint32_t rank,
                                                 int& m0, int& n0) {
    const int tiles_mc = (prm.tiles_m + 1) / 2;
    const int gm = prm.group_m / 2 > 0 ? prm.group_m / 2 : 1;
    const int in_group = gm * prm.tiles_n;
    const int first_m = (pid / in_group) * gm;
    const int gsz = min(tiles_mc - first_m, gm);
    const int local = pid % in_group;
    m0 = ((first_m + local % gsz) * 2 + (int)rank) * kTM;
    n0 = (local / gsz) * kTN;
}

__global__ void __launch_bounds__(kPairThreads, 1)
    emul_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA,
                          const __grid_constant__ CUtensorMap tmB, EmulGemmParams prm) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw_u32 = smem_u32(smem_raw);
    unsigned char* smem = smem_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
    unsigned char* tiles = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kPairStages * kPairStageBytes);
    uint64_t* empty = full + kPairStages;
    uint64_t* accf = empty + kPairStages;
    uint64_t* acce = accf + 2;
    uint64_t* done = acce + 2;
    uint64_t* agg = done + 1;   // block 1: its epilogue warps' hand-backs, gathered
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(agg + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* njobs_slot = const_cast<int*>(reinterpret_cast<volatile int*>(abort_flag + 1));
    uint32_t* jobs = reinterpret_cast<uint32_t*>(smem + kPairStages * kPairStageBytes + 256);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kPairStages; ++i) {
            mbar_init(&full[i], 1);    // block 0's producer; bytes of both blocks
            mbar_init(&empty[i], 1);   // one multicast commit per round
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 2 * kEpiWarps);   // epilogue warps of both blocks
            mbar_init(&agg[b], kEpiWarps);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        // the tail split counts clusters: both blocks of a pair take the same piece
        int t_lo = 2, t_hi = prm.s + 1;
        const int cid = (int)blockIdx.x / 2;
        if (cid >= prm.n_full) {
            const int pc = (cid - prm.n_full) % prm.pieces;
            const uint32_t r = (uint32_t)(prm.t_ranges >> (8 * pc)) & 0xffu;
            t_lo = (int)(r & 15u) + 2;
            t_hi = (int)(r >> 4) + 2;
        }
        *njobs_slot = build_jobs(prm.s, (int)prm.K, prm.digit_bits, prm.trim != 0, prm.crt != 0,
                                 t_lo, t_hi, jobs);
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc_pair(tmem_slot, kTmemCols);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    cluster_sync_all();   // both blocks' barriers and TMEM exist before any signal
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int njobs = *njobs_slot;

    int m0, n0;
    {
        const int cid = (int)blockIdx.x / 2;
        const int pid = cid < prm.n_full ? cid : prm.n_full + (cid - prm.n_full) / prm.pieces;
        pair_tile_origin(prm, pid, rank, m0, n0);
    }
    const uint64_t tmo = prm.timeout_ns;
    const uint32_t full0 = cluster_addr(full, 0);   // block 0's full barriers
    // each warpgroup changes its registers once, before its warps part: the
    // epilogue's (warps 4-11) take what warps 0-3 and 12-15 give back
    const int wg = warp >> 2;
    if (wg == 1 || wg == 2) {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kPairEpiRegs));
        epilogue_role(prm, jobs, njobs, tmem_base, accf, &acce[0],
                      leader ? 0u : cluster_addr(acce, 0), agg, m0, n0, warp, lane, tmo,
                      abort_flag, warp - 4);
    } else {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kPairLowRegs));
    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both blocks) ----------------
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
            uint32_t it = 0;
            bool ok = true;
            for (int j = 0; j < njobs && ok; ++j) {
                const uint32_t jd = jobs[j];
                for (int kb = job_kb(jd); kb < job_ke(jd); ++kb, ++it) {
                    const uint32_t st = it % kPairStages, round = it / kPairStages;
                    if (it >= (uint32_t)kPairStages &&
                        !mbar_wait_bounded(&empty[st], (round - 1) & 1, tmo, abort_flag, prm.err)) {
                        ok = false;
                        break;
                    }
                    if (leader) mbar_arrive_expect_tx(&full[st], 2 * kPairStageBytes);
                    // fault injection: block 0 issues no copy, the stage never fills
                    if ((int64_t)it == prm.inject_skip_it && blockIdx.x == 0) continue;
                    unsigned char* a = tiles + st * kPairStageBytes;
                    tma_load_3d_pair(a, &tmA, full0 + st * 8, kb * kTK, m0, job_p(jd) - 1);
                    tma_load_3d_pair(a + kATile, &tmB, full0 + st * 8, kb * kTK,
                                     n0 + (int)rank * (kTN / 2), job_q(jd) - 1);
                }
            }
            // The MMAs of every issued stage must have consumed it (so this
            // block's copies have landed, on block 0's barrier) and its
            // release reached this block.  After an abort (this block's, or a
            // timeout recorded by any block) the stages not consumed are never
            // released: their copies were issued before the abort was seen and
            // land within microseconds, so those waits are cut to kDrainNs.
            const bool aborted =
                *abort_flag ||
                (prm.err && *reinterpret_cast<volatile int*>(prm.err) == ALP_ERR_TIMEOUT);
            const uint64_t drain = aborted && tmo > kDrainNs ? kDrainNs : tmo;
            for (uint32_t j = it > (uint32_t)kPairStages ? it - kPairStages : 0; j < it; ++j)
                if (!mbar_wait_bounded(&empty[j % kPairStages], (j / kPairStages) & 1, drain,
                                       nullptr, prm.err, false) &&
                    aborted)
                    break;   // not consumed; neither is any later stage
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---------------- MMA issuer (block 0) ----------------
            const uint32_t idesc = idesc_bf16_f32(2 * kTM, kTN);
            uint32_t it = 0;
            bool ok = true;
            for (int job = 0; job < njobs && ok; ++job) {
                const uint32_t jd = jobs[job];
                const uint32_t b = job & 1;
                if (job >= 2 &&
                    !mbar_wait_bounded(&acce[b], ((job >> 1) - 1) & 1, tmo, abort_flag, prm.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + b * kTN;
                uint32_t accumulate = 0;
                for (int kb = job_kb(jd); kb < job_ke(jd); ++kb, ++it) {
                    const uint32_t st = it % kPairStages, round = it / kPairStages;
                    if (!mbar_wait_bounded(&full[st], round & 1, tmo, abort_flag, prm.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(tiles + st * kPairStageBytes);
                    const uint64_t adesc = sw128_kmajor_desc(a_addr);
                    const uint64_t bdesc = sw128_kmajor_desc(a_addr + kATile);
#pragma unroll
                    for (int kk = 0; kk < kTK / 16; ++kk) {
                        umma_bf16_pair(d_tmem, adesc + 2 * kk, bdesc + 2 * kk, idesc, accumulate);
                        accumulate = 1;
                    }
                    umma_commit_pair(&empty[st], 3);
                }
                if (!ok) break;
                umma_commit_pair(&accf[b], 3);
            }
            // all MMAs must have completed before TMEM and shared memory go away,
            // and both blocks' hand-backs of the last two chunks must have
            // arrived.  After an abort the epilogue warps leave without handing
            // back; an arrival block 1 did send precedes its cluster barrier
            // arrival, which block 0 waits for before it exits.
            umma_commit_pair(done, 1);
            mbar_wait_bounded(done, 0, tmo, nullptr, prm.err, false);
            for (int job = njobs > 2 ? njobs - 2 : 0; job < njobs && ok; ++job)
                mbar_wait_bounded(&acce[job & 1], (job >> 1) & 1, tmo, nullptr, prm.err, false);
        }
    }
    }   // warps 2, 3 and 12-15 have no role
    tc_fence_before();
    __syncwarp();
    cluster_sync_all();   // no block leaves while its peer's MMAs or signals may reach it
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, kTmemCols);
    }
}


// ---------------------------------------------------------------------------
// The modular scheme with the reconstruction in the product kernel.
//
// A persistent launch of CTA pairs (P clusters, all resident) that take
// items from a counter as they go, an item being a whole 256 x 256 tile (all
// n moduli; items 0..n_full-1 in raster order) or one piece of a tail tile (a
// range of moduli; tail_split).  Block 0's producer takes the cluster's next
// item when it has issued the copies of the current one and publishes it in
// the cluster's list in global memory; every other role of both blocks reads
// the list (bounded waits), so that a pair that runs faster takes more items
// and the launch ends evenly.  The producer, the MMA issuer and the epilogue walk the
// same items and, per item, the moduli and 1024-k chunks in order, so the
// stage ring and the accumulator double buffer run on across items as within
// one.  Sixteen warps per block: 0 the TMA producer, 1 the MMA issuer, 4-11
// the epilogue (the drains, hand-backs and residue bytes of
// emul_gemm_pair_kernel), 12-15 the reconstruction; 2-3 idle.  When the
// epilogue has stored the last residue plane of a whole tile it counts the
// tile in shared memory (a release add per warp); the reconstruction warps
// wait for the count (bounded) and rebuild the block's 128 rows of that tile
// from its n byte planes, as the standalone kernels do, while the next
// tile's products run, so that C is written during the products instead of
// by a launch of its own.  Tail tiles (whose moduli several clusters share)
// are reconstructed by crt_tail_recombine_kernel after the launch.
// Registers: the epilogue's warpgroups take 176 per thread, the others give
// theirs down to 80 (setmaxnreg): 2 x 128 x 176 + 2 x 128 x 80 = 65536, the
// 512 threads x 128 registers of the launch.
// ---------------------------------------------------------------------------
struct CrtFuse {
    const int32_t* e;   // exponents of the rows of op(A) (M)
    const int32_t* f;   // exponents of the columns of op(B) (N)
    double alpha, beta;
    double* C;
    int64_t ldc;
    int amode;          // alpha: 0 one, 1 minus one, 2 any
    int bmode;          // beta: 0 zero (C not read), 1 any
    int n_items;        // whole tiles n_full, then (pair tiles - n_full) * pieces
    // the schedule (workspace, all bytes 0xff before the launch): sched[0] the
    // item counter, sched[1 + c * stride + k] the k-th item of cluster c
    // (n_items or more: no more items), stride = n_items + 1
    int* sched;
    int stride;
    CrtRecConsts cc;
};
constexpr int kFusedThreads = 512;
constexpr int kFusedEpiWarp0 = 4;    // warps 4..11: epilogue
constexpr int kFusedRecWarp0 = 12;   // warps 12..15: reconstruction
constexpr int kFusedEpiRegs = 176, kFusedLowRegs = 80;
constexpr int kMaxFusedClusters = 128;   // clusters of one launch (the schedule's bound)
static_assert(2 * 128 * kFusedEpiRegs + 2 * 128 * kFusedLowRegs == kFusedThreads * 128,
              "register split of the fused kernel");

// Item i: the pair tile and its moduli q_lo..q_hi (planes, 0-based).
__device__ __forceinline__ void fused_item(const EmulGemmParams& prm, int i, int& pid, int& q_lo,
                                           int& q_hi) {
    if (i < prm.n_full) {
        pid = i;
        q_lo = 0;
        q_hi = prm.s - 1;
        return;
    }
    const int pc = (i - prm.n_full) % prm.pieces;
    pid = prm.n_full + (i - prm.n_full) / prm.pieces;
    const uint32_t r = (uint32_t)(prm.t_ranges >> (8 * pc)) & 0xffu;
    q_lo = (int)(r & 15u);
    q_hi = (int)(r >> 4);
}

// The k-th item of cluster c: block 0's producer takes it from the counter
// and publishes it (fused_take); the other roles wait for it (fused_next).
__device__ __forceinline__ int fused_take(const CrtFuse& fz, int c, int k) {
    int item = (int)(atomicAdd(reinterpret_cast<unsigned int*>(fz.sched), 1u) + 1u);
    if (item > fz.n_items || item < 0) item = fz.n_items;
    *reinterpret_cast<volatile int*>(fz.sched + 1 + (int64_t)c * fz.stride + k) = item;
    return item;
}
__device__ __forceinline__ int fused_next(const CrtFuse& fz, int c, int k, uint64_t limit_ns,
                                          volatile int* abort, int* err) {
    const volatile int* p = fz.sched + 1 + (int64_t)c * fz.stride + k;
    int v = *p;
    if (v != -1) return v;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1;; ++i) {
        __nanosleep(64);
        v = *p;
        if (v != -1) return v;
        if (abort && *abort) return fz.n_items;
        if ((i & 15u) != 0) continue;
        if (err && *reinterpret_cast<volatile int*>(err) == ALP_ERR_TIMEOUT) {
            if (abort) *abort = 1;
            return fz.n_items;
        }
        if (globaltimer() - t0 > limit_ns) {
            set_device_error(err, ALP_ERR_TIMEOUT);
            if (abort) *abort = 1;
            return fz.n_items;
        }
    }
}

// C at row i, columns j..j+3 from the n byte planes of prm.G (one 32-bit load
// per plane: crt_fused_load), as the standalone kernels form it (crt_rec.cuh),
// stored with alpha and beta (crt_fused_finish).  Rows past M and columns
// past N are skipped.
__device__ __forceinline__ void crt_fused_load(const EmulGemmParams& prm, int64_t i, int64_t j,
                                               uint32_t (&v)[16]) {
    const bool in = i < prm.M && j < prm.N;
    const uint8_t* g = reinterpret_cast<const uint8_t*>(prm.G) + i * prm.ldg + j;
#pragma unroll
    for (int l = 0; l < 16; ++l)
        v[l] = (in && l < prm.s)
                   ? __ldcg(reinterpret_cast<const unsigned int*>(g + (int64_t)l * prm.gplane))
                   : 0u;
}
__device__ __forceinline__ void crt_fused_finish(const EmulGemmParams& prm, const CrtFuse& fz,
                                                 int64_t i, int64_t j, const uint32_t (&v)[16]) {
    if (i >= prm.M || j >= prm.N) return;
    int64_t hi[4];
    uint64_t lo[4];
    crt_reconstruct4_n(v, prm.s, fz.cc, hi, lo);
    const int ei = __ldg(fz.e + i) - 2 * fz.cc.k;
    const bool full = j + 3 < prm.N;
    double* ci = fz.C + i * fz.ldc + j;
    double o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        // a column past N computes from the padding bytes and is not stored
        const int fj = (full || j + u < prm.N) ? __ldg(fz.f + j + u) : 0;
        const double w = i128_scaled_to_double_rn(hi[u], lo[u], ei + fj);
        o[u] = fz.amode == 0 ? w : fz.amode == 1 ? -w : fz.alpha * w;
    }
    if (fz.bmode) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (full || j + u < prm.N) o[u] = __fma_rn(fz.beta, ci[u], o[u]);
    }
    if (full && (reinterpret_cast<uintptr_t>(ci) & 15) == 0) {
        reinterpret_cast<double2*>(ci)[0] = make_double2(o[0], o[1]);
        reinterpret_cast<double2*>(ci)[1] = make_double2(o[2], o[3]);
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (full || j + u < prm.N) ci[u] = o[u];
    }
}

__device__ __forceinline__ uint32_t ld_acquire_cta(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_cta_add(uint32_t* p, uint32_t v) {
    asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v)
                 : "memory");
}
// Waits until *cnt >= target, as mbar_wait_bounded waits for a phase (gives
// up after limit_ns, at once when the block aborts or a timeout was recorded
// anywhere; records ALP_ERR_TIMEOUT when its own limit runs out).  Sleeps
// between polls: a tile's products take hundreds of microseconds.
__device__ __forceinline__ bool count_wait_bounded(const uint32_t* cnt, uint32_t target,
                                                   uint64_t limit_ns, volatile int* abort,
                                                   int* err) {
    if (ld_acquire_cta(cnt) >= target) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1;; ++i) {
        __nanosleep(512);
        if (ld_acquire_cta(cnt) >= target) return true;
        if (*abort) return false;
        if ((i & 15u) != 0) continue;
        if (err && *reinterpret_cast<volatile int*>(err) == ALP_ERR_TIMEOUT) {
            *abort = 1;
            return false;
        }
        if (globaltimer() - t0 > limit_ns) {
            set_device_error(err, ALP_ERR_TIMEOUT);
            *abort = 1;
            return false;
        }
    }
}

// The epilogue warps of the fused kernel (4..11): the drains, hand-backs and
// residue bytes of every modulus as epilogue_role has them; after the last
// modulus of a whole tile each warp counts it in tiles_ready (release).
__device__ __forceinline__ void fused_epilogue(const EmulGemmParams& prm, const CrtFuse& fz,
                                               uint32_t tmem_base, uint64_t* accf,
                                               uint64_t* acce, uint32_t acce_remote,
                                               uint64_t* agg, uint32_t* tiles_ready,
                                               uint32_t rank, int warp, int lane, uint64_t tmo,
                                               volatile int* abort_flag) {
    const int quarter = warp & 3;                      // TMEM lanes this warp may access
    const int half = (warp - kFusedEpiWarp0) >> 2;     // columns [128*half, 128*half + 128)
    const int row = quarter * 32 + lane;
    const int kblocks = (int)((prm.K + kTK - 1) / kTK), cpm = (kblocks + 15) / 16;
    uint32_t acc[128];
    int job = 0;
    bool ok = true;
    const int cid = (int)blockIdx.x / 2;
    for (int k = 0; ok && k < fz.stride; ++k) {
        const int it = fused_next(fz, cid, k, tmo, abort_flag, prm.err);
        if (it >= fz.n_items) break;
        int pid, qlo, qhi, m0, n0;
        fused_item(prm, it, pid, qlo, qhi);
        pair_tile_origin(prm, pid, rank, m0, n0);
        const int gm = m0 + row;
        for (int q = qlo; q <= qhi && ok; ++q) {
#pragma unroll
            for (int x = 0; x < 128; ++x) acc[x] = 0;
            for (int c = 0; c < cpm; ++c, ++job) {
                const uint32_t b = job & 1;
                if (!mbar_wait_bounded(&accf[b], (job >> 1) & 1, tmo, abort_flag, prm.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr =
                    tmem_base + ((uint32_t)(quarter * 32) << 16) + b * kTN + half * 128;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) tmem_drain32_cvt(taddr + cc * 32, &acc[cc * 32]);
                tc_fence_before();
                __syncwarp();
                // the first epilogue warp forwards block 1's hand-backs
                if (lane == 0)
                    hand_back(acce, acce_remote, agg, b, job, warp - kFusedEpiWarp0 + 2, tmo,
                              abort_flag, prm.err);
            }
            if (!ok) break;
            // plane q receives x = (Q y_q) mod m_q, one byte per column
            const uint32_t m = crt_modulus(q), magic = crt_magic(m), y = prm.crt_y[q];
            uint8_t* g = reinterpret_cast<uint8_t*>(prm.G) + (int64_t)q * prm.gplane +
                         (int64_t)gm * prm.ldg + n0 + half * 128;
            if (gm < prm.M) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    uint32_t w[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = 16 * i + 4 * u;
                        w[u] = crt_mod(crt_residue((int32_t)acc[c], m, magic) * y, m, magic) |
                               crt_mod(crt_residue((int32_t)acc[c + 1], m, magic) * y, m, magic)
                                   << 8 |
                               crt_mod(crt_residue((int32_t)acc[c + 2], m, magic) * y, m, magic)
                                   << 16 |
                               crt_mod(crt_residue((int32_t)acc[c + 3], m, magic) * y, m, magic)
                                   << 24;
                    }
                    *reinterpret_cast<uint4*>(g + 16 * i) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        }
        if (ok && it < prm.n_full) {
            // every plane of this whole tile is stored: count it
            __threadfence_block();
            __syncwarp();
            if (lane == 0) red_release_cta_add(tiles_ready, 1u);
        }
    }
}

// The reconstruction warps (12..15, 128 threads): the whole tiles of this
// cluster in order, each once all eight epilogue warps have counted it; four
// columns per thread, 64 threads per row, two rows per step (64 steps for the
// block's 128 rows), with the lines of the step after next asked of L2.
__device__ __forceinline__ void fused_reconstruction(const EmulGemmParams& prm, const CrtFuse& fz,
                                                     const uint32_t* tiles_ready, uint32_t rank,
                                                     int warp, int lane, uint64_t tmo,
                                                     volatile int* abort_flag) {
    const int rt = (int)threadIdx.x - 32 * kFusedRecWarp0;   // 0..127
    const int w = warp - kFusedRecWarp0;                     // 0..3
    const int cid = (int)blockIdx.x / 2;
    uint32_t k = 0;   // whole tiles of this cluster so far
    for (int x = 0; x < fz.stride; ++x) {
        const int it = fused_next(fz, cid, x, tmo, abort_flag, prm.err);
        if (it >= fz.n_items) return;
        if (it >= prm.n_full) continue;   // a tail piece: reconstructed after the launch
        ++k;
        if (!count_wait_bounded(tiles_ready, (uint32_t)(kEpiWarps) * k, tmo, abort_flag, prm.err))
            return;
        int m0, n0;
        pair_tile_origin(prm, it, rank, m0, n0);
        const int64_t j = (int64_t)n0 + 4 * (rt & 63);
#pragma unroll 1
        for (int step = 0; step < 64; ++step) {
            if (step + 2 < 64 && lane < prm.s) {
                const int64_t ip = (int64_t)m0 + 2 * (step + 2) + (w >> 1);
                if (ip < prm.M)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(
                        reinterpret_cast<const uint8_t*>(prm.G) + (int64_t)lane * prm.gplane +
                        ip * prm.ldg + n0 + 128 * (w & 1)));
            }
            const int64_t i = (int64_t)m0 + 2 * step + (rt >> 6);
            uint32_t v[16];
            crt_fused_load(prm, i, j, v);
            crt_fused_finish(prm, fz, i, j, v);
        }
    }
}

__global__ void __launch_bounds__(kFusedThreads, 1)
    emul_crt_fused_pair_kernel(const __grid_constant__ CUtensorMap tmA,
                               const __grid_constant__ CUtensorMap tmB, EmulGemmParams prm,
                               CrtFuse fz) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw_u32 = smem_u32(smem_raw);
    unsigned char* smem = smem_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
    unsigned char* tiles = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kPairStages * kPairStageBytes);
    uint64_t* empty = full + kPairStages;
    uint64_t* accf = empty + kPairStages;
    uint64_t* acce = accf + 2;
    uint64_t* done = acce + 2;
    uint64_t* agg = done + 1;    // block 1: its epilogue warps' hand-backs, gathered
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(agg + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint32_t* tiles_ready = tmem_slot + 2;   // whole tiles stored, times kEpiWarps

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kPairStages; ++i) {
            mbar_init(&full[i], 1);    // block 0's producer; bytes of both blocks
            mbar_init(&empty[i], 1);   // one multicast commit per round
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 2 * kEpiWarps);   // epilogue warps of both blocks
            mbar_init(&agg[b], kEpiWarps);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *tiles_ready = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc_pair(tmem_slot, kTmemCols);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    cluster_sync_all();   // both blocks' barriers and TMEM exist before any signal
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint64_t tmo = prm.timeout_ns;
    const uint32_t full0 = cluster_addr(full, 0);   // block 0's full barriers
    const int kblocks = (int)((prm.K + kTK - 1) / kTK), cpm = (kblocks + 15) / 16;
    const int cid = (int)blockIdx.x / 2;

    // each warpgroup changes its registers once, before its warps part: the
    // epilogue's (1, 2) take what the others (0, 3) give back
    const int wg = warp >> 2;
    if (wg == 1 || wg == 2) {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kFusedEpiRegs));
        fused_epilogue(prm, fz, tmem_base, accf, &acce[0], leader ? 0u : cluster_addr(acce, 0),
                       agg, tiles_ready, rank, warp, lane, tmo, abort_flag);
    } else if (wg == 3) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kFusedLowRegs));
        fused_reconstruction(prm, fz, tiles_ready, rank, warp, lane, tmo, abort_flag);
    } else {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kFusedLowRegs));
    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both blocks) ----------------
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
            uint32_t it = 0;
            bool ok = true;
            for (int k = 0; ok && k < fz.stride; ++k) {
                const int item = leader ? fused_take(fz, cid, k)
                                        : fused_next(fz, cid, k, tmo, abort_flag, prm.err);
                if (item >= fz.n_items) break;
                int pid, qlo, qhi, m0, n0;
                fused_item(prm, item, pid, qlo, qhi);
                pair_tile_origin(prm, pid, rank, m0, n0);
                for (int q = qlo; q <= qhi && ok; ++q) {
                    for (int kb = 0; kb < kblocks; ++kb, ++it) {
                        const uint32_t st = it % kPairStages, round = it / kPairStages;
                        if (it >= (uint32_t)kPairStages &&
                            !mbar_wait_bounded(&empty[st], (round - 1) & 1, tmo, abort_flag,
                                               prm.err)) {
                            ok = false;
                            break;
                        }
                        if (leader) mbar_arrive_expect_tx(&full[st], 2 * kPairStageBytes);
                        // fault injection: block 0 issues no copy, the stage never fills
                        if ((int64_t)it == prm.inject_skip_it && blockIdx.x == 0) continue;
                        unsigned char* a = tiles + st * kPairStageBytes;
                        tma_load_3d_pair(a, &tmA, full0 + st * 8, kb * kTK, m0, q);
                        tma_load_3d_pair(a + kATile, &tmB, full0 + st * 8, kb * kTK,
                                         n0 + (int)rank * (kTN / 2), q);
                    }
                }
            }
            // as in emul_gemm_pair_kernel: every issued stage consumed and
            // released before this block leaves (cut to kDrainNs after an abort)
            const bool aborted =
                *abort_flag ||
                (prm.err && *reinterpret_cast<volatile int*>(prm.err) == ALP_ERR_TIMEOUT);
            const uint64_t drain = aborted && tmo > kDrainNs ? kDrainNs : tmo;
            for (uint32_t j = it > (uint32_t)kPairStages ? it - kPairStages : 0; j < it; ++j)
                if (!mbar_wait_bounded(&empty[j % kPairStages], (j / kPairStages) & 1, drain,
                                       nullptr, prm.err, false) &&
                    aborted)
                    break;
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---------------- MMA issuer (block 0) ----------------
            const uint32_t idesc = idesc_bf16_f32(2 * kTM, kTN);
            uint32_t it = 0;
            int job = 0;
            bool ok = true;
            for (int k = 0; ok && k < fz.stride; ++k) {
                const int item = fused_next(fz, cid, k, tmo, abort_flag, prm.err);
                if (item >= fz.n_items) break;
                int pid, qlo, qhi;
                fused_item(prm, item, pid, qlo, qhi);
                for (int q = qlo; q <= qhi && ok; ++q) {
                    for (int c = 0; c < cpm && ok; ++c, ++job) {
                        const uint32_t b = job & 1;
                        if (job >= 2 && !mbar_wait_bounded(&acce[b], ((job >> 1) - 1) & 1, tmo,
                                                           abort_flag, prm.err)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d_tmem = tmem_base + b * kTN;
                        uint32_t accumulate = 0;
                        const int ke = 16 * c + 16 < kblocks ? 16 * c + 16 : kblocks;
                        for (int kb = 16 * c; kb < ke; ++kb, ++it) {
                            const uint32_t st = it % kPairStages, round = it / kPairStages;
                            if (!mbar_wait_bounded(&full[st], round & 1, tmo, abort_flag,
                                                   prm.err)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t a_addr = smem_u32(tiles + st * kPairStageBytes);
                            const uint64_t adesc = sw128_kmajor_desc(a_addr);
                            const uint64_t bdesc = sw128_kmajor_desc(a_addr + kATile);
#pragma unroll
                            for (int kk = 0; kk < kTK / 16; ++kk) {
                                umma_bf16_pair(d_tmem, adesc + 2 * kk, bdesc + 2 * kk, idesc,
                                               accumulate);
                                accumulate = 1;
                            }
                            umma_commit_pair(&empty[st], 3);
                        }
                        if (!ok) break;
                        umma_commit_pair(&accf[b], 3);
                    }
                }
            }
            // as in emul_gemm_pair_kernel: all MMAs complete and both blocks'
            // hand-backs of the last two chunks arrived
            umma_commit_pair(done, 1);
            mbar_wait_bounded(done, 0, tmo, nullptr, prm.err, false);
            for (int j = job > 2 ? job - 2 : 0; j < job && ok; ++j)
                mbar_wait_bounded(&acce[j & 1], (j >> 1) & 1, tmo, nullptr, prm.err, false);
        }
    }
    }   // warpgroup 0; warps 2 and 3 have no role
    tc_fence_before();
    __syncwarp();
    cluster_sync_all();   // no block leaves while its peer's MMAs or signals may reach it
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, kTmemCols);
    }
}

// The tail tiles of a fused launch (pair tiles n_full..): 16 blocks of 256
// threads per tile, block b holding rows 16 (b % 8) .. + 16 of the tile's
// half (b / 8) % 2, four rows per step.
__global__ void __launch_bounds__(256) crt_tail_recombine_kernel(EmulGemmParams prm, CrtFuse fz) {
    const int b = (int)blockIdx.x;
    const int strip = b & 7, r = (b >> 3) & 1, pid = prm.n_full + (b >> 4);
    int m0, n0;
    pair_tile_origin(prm, pid, (uint32_t)r, m0, n0);
    const int64_t j = (int64_t)n0 + 4 * (threadIdx.x & 63);
#pragma unroll 1
    for (int step = 0; step < 4; ++step) {
        const int64_t i = (int64_t)m0 + 16 * strip + 4 * step + (threadIdx.x >> 6);
        uint32_t v[16];
        crt_fused_load(prm, i, j, v);
        crt_fused_finish(prm, fz, i, j, v);
    }
}

}  // namespace

// Tail split of a launch of `tiles` tiles on `sms` SMs (one block each): the
// last, partial wave of r tiles becomes r * pieces blocks, pieces = the
// largest count <= min(sms / r, s, 8) whose best cut of groups t = 2..s+1
// (group t holds t-1 digit pairs) into contiguous ranges keeps the largest
// piece smallest.  No split when the last wave is full or pieces < 2.
TailSplit tail_split(int tiles, int s, int sms, bool trim, bool crt) {
    TailSplit ts;
    ts.n_full = tiles;
    ts.pieces = 1;
    for (int i = 0; i < 8; ++i) ts.t_lo[i] = ts.t_hi[i] = 0;
    ts.t_lo[0] = 2;
    ts.t_hi[0] = s + 1;
    if (tiles <= 0 || sms <= 0 || s < 2) return ts;
    const int r = tiles % sms == 0 ? sms : tiles % sms;
    int k = sms / r;
    if (k > s) k = s;
    if (k > 8) k = 8;
    if (k < 2 || r == sms) return ts;
    // smallest threshold whose greedy contiguous cut needs <= k pieces; group t
    // holds t-1 pairs (2 when it is the trimmed last group)
    auto weight = [&](int t) { return crt ? 1 : (trim && t == s + 1 && s > 2) ? 2 : t - 1; };
    int total = 0, widest = 0;
    for (int t = 2; t <= s + 1; ++t) {
        total += weight(t);
        widest = weight(t) > widest ? weight(t) : widest;
    }
    for (int cap = widest; cap <= total; ++cap) {
        int lo[8], hi[8], n = 0, acc = 0;
        bool fits = true;
        for (int t = 2; t <= s + 1 && fits; ++t) {
            const int w = weight(t);
            if (n == 0 || acc + w > cap) {
                if (n == k) fits = false;
                else {
                    lo[n] = t;
                    hi[n] = t;
                    ++n;
                    acc = w;
                }
            } else {
                hi[n - 1] = t;
                acc += w;
            }
        }
        if (!fits) continue;
        ts.n_full = tiles - r;
        ts.pieces = n;
        for (int i = 0; i < n; ++i) {
            ts.t_lo[i] = lo[i];
            ts.t_hi[i] = hi[i];
        }
        if (n < 2) ts.n_full = tiles;
        return ts;
    }
    return ts;
}

alp_status emul_slice_gemm(int64_t M, int64_t N, int64_t K, int s, const __nv_bfloat16* da,
                           const __nv_bfloat16* db, int64_t kpad, int32_t* G, int64_t ldg,
                           cudaStream_t stream, int group_m, int cluster, int digit_bits,
                           bool trim, bool crt) {
    if (crt) {
        if (s < kCrtMinModuli || s > kCrtMaxModuli || K > kCrtMaxK) return ALP_ERR_UNSUPPORTED;
    } else if (!emul_digit_bits_ok(digit_bits) || s > emul_max_slices(digit_bits) ||
               K > emul_max_k(digit_bits)) {
        return ALP_ERR_UNSUPPORTED;
    }
    {   // the job table of one tile must fit its shared-memory slot
        const int64_t kblocks = (K + kTK - 1) / kTK;
        int64_t njobs = crt ? s * ((kblocks + 1024 / kTK - 1) / (1024 / kTK)) : 0;
        for (int t = 2; t <= s + 1 && !crt; ++t)
            for (int pp = (t - s > 1 ? t - s : 1); pp <= (s < t - 1 ? s : t - 1); ++pp) {
                const int qq = t - pp;
                if (!emul_pair_kept(pp, qq, s, trim)) continue;
                const int64_t cb = chunk_of(pp, qq, digit_bits) / kTK;
                njobs += (kblocks + cb - 1) / cb;
            }
        if (njobs > kMaxJobs || kblocks > 1023) return ALP_ERR_UNSUPPORTED;
    }
    const int arr = (cluster == kEmulSingle || cluster == kEmulPair) ? cluster : emul_cluster();
    const int cl = arr == kEmulSingle ? 1 : 2;   // blocks per cluster
    CUtensorMap ta, tb;
    alp_status st = make_tmap_3d_bf16(&ta, da, (uint64_t)kpad, (uint64_t)M, (uint64_t)s, kTK, kTM);
    if (st != ALP_OK) return st;
    st = make_tmap_3d_bf16(&tb, db, (uint64_t)kpad, (uint64_t)N, (uint64_t)s, kTK, kTN / cl);
    if (st != ALP_OK) return st;
    EmulGemmParams p;
    p.M = M;
    p.N = N;
    p.K = K;
    p.s = s;
    p.digit_bits = digit_bits;
    p.trim = trim ? 1 : 0;
    p.crt = crt ? 1 : 0;
    for (int l = 0; l < kCrtMaxModuli; ++l) p.crt_y[l] = crt && l < s ? crt_weight(s, l) : 0;
    p.G = G;
    p.ldg = ldg;
    p.gplane = M * ldg;
    const int64_t tiles_m = (M + kTM - 1) / kTM, tiles_n = (N + kTN - 1) / kTN;
    if (tiles_m * tiles_n > 0x7fffffff) return ALP_ERR_UNSUPPORTED;
    p.tiles_m = (int)tiles_m;
    p.tiles_n = (int)tiles_n;
    p.group_m = group_m > 0 ? group_m : emul_group_m(arr == kEmulPair);
    p.timeout_ns = wait_timeout_ns();
    p.err = device_error_word();
    p.inject_skip_it = inject_skip_kt();
    const int tiles = (int)(tiles_m * tiles_n);
    p.n_full = 0x7fffffff;   // every block a whole tile unless split below
    p.pieces = 1;
    p.t_ranges = (uint64_t)(s - 1) << 4;
    if (cl == 1 && emul_tail_split_on()) {
        const TailSplit ts = tail_split(tiles, s, device_sm_count(), trim, crt);
        p.n_full = ts.n_full;
        p.pieces = ts.pieces;
        p.t_ranges = 0;
        for (int i = 0; i < ts.pieces; ++i)
            p.t_ranges |= (uint64_t)((ts.t_lo[i] - 2) | (ts.t_hi[i] - 2) << 4) << (8 * i);
    }
    if (cl == 1) {
        const int64_t grid = p.n_full >= tiles
                                 ? (int64_t)tiles
                                 : (int64_t)p.n_full + (int64_t)(tiles - p.n_full) * p.pieces;
        cudaError_t e = cudaFuncSetAttribute(emul_gemm_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return cuda_status(e);
        emul_gemm_kernel<<<(unsigned)grid, kThreads, kSmemBytes, stream>>>(ta, tb, p);
        return cuda_status(cudaGetLastError());
    }
    const int smem_bytes = kPairSmemBytes;
    const int64_t pair_tiles = ((tiles_m + 1) / 2) * tiles_n;
    int64_t clusters = pair_tiles;
    if (emul_tail_split_on()) {   // in units of pairs, half the SMs each
        const TailSplit ts = tail_split((int)pair_tiles, s, device_sm_count() / 2, trim, crt);
        p.n_full = ts.n_full;
        p.pieces = ts.pieces;
        p.t_ranges = 0;
        for (int i = 0; i < ts.pieces; ++i)
            p.t_ranges |= (uint64_t)((ts.t_lo[i] - 2) | (ts.t_hi[i] - 2) << 4) << (8 * i);
        if (ts.n_full < pair_tiles) clusters = ts.n_full + (pair_tiles - ts.n_full) * ts.pieces;
    }
    cudaError_t e = cudaFuncSetAttribute(emul_gemm_pair_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return cuda_status(e);
    const int64_t grid = 2 * clusters;
    if (grid > 0x7fffffff) return ALP_ERR_UNSUPPORTED;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(kPairThreads);
    lc.dynamicSmemBytes = smem_bytes;
    lc.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    e = cudaLaunchKernelEx(&lc, emul_gemm_pair_kernel, ta, tb, p);
    return cuda_status(e);
}

// Clusters of the fused kernel that are resident at once (its persistent
// grid); half the SMs if the query fails.
static int fused_active_clusters() {
    static int c = 0;
    if (c == 0) {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)(2 * device_sm_count()));
        lc.blockDim = dim3(kFusedThreads);
        lc.dynamicSmemBytes = kFusedSmemBytes;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, emul_crt_fused_pair_kernel, &lc) != cudaSuccess ||
            nc < 1) {
            (void)cudaGetLastError();
            nc = device_sm_count() / 2;
        }
        c = nc > 0 ? nc : 1;
    }
    return c;
}

size_t emul_crt_sched_bytes(int64_t M, int64_t N) {
    if (M <= 0 || N <= 0) return 0;
    const int64_t pair_tiles = ((M + 2 * kTM - 1) / (2 * kTM)) * ((N + kTN - 1) / kTN);
    return (size_t)4 * (1 + (size_t)kMaxFusedClusters * (size_t)(pair_tiles + 7 * kMaxFusedClusters + 1));
}

alp_status emul_crt_products_recombine(int64_t M, int64_t N, int64_t K, int n,
                                       const __nv_bfloat16* da, const __nv_bfloat16* db,
                                       int64_t kpad, uint8_t* G, int64_t ldg, const int32_t* e,
                                       const int32_t* f, int k, double alpha, double beta,
                                       double* C, int64_t ldc, int* sched, size_t sched_bytes,
                                       cudaStream_t stream, int group_m, int cluster, int fuse) {
    if (n < kCrtMinModuli || n > kCrtMaxModuli || K > kCrtMaxK || k < 1 || k > 60)
        return ALP_ERR_UNSUPPORTED;
    const int arr = (cluster == kEmulSingle || cluster == kEmulPair) ? cluster : emul_cluster();
    const bool fused = fuse > 0 || (fuse < 0 && emul_crt_fuse_on());
    if (arr != kEmulPair || !fused || !sched || sched_bytes < emul_crt_sched_bytes(M, N)) {
        alp_status st = emul_slice_gemm(M, N, K, n, da, db, kpad, reinterpret_cast<int32_t*>(G),
                                        ldg, stream, group_m, arr, kDigitBits, false, true);
        if (st != ALP_OK) return st;
        return launch_recombine_crt(n, k, recombine_grid(M, N), stream, G, M * ldg, ldg, e, f, M,
                                    N, alpha, beta, C, ldc);
    }
    if ((K + kTK - 1) / kTK > 1023) return ALP_ERR_UNSUPPORTED;
    CUtensorMap ta, tb;
    alp_status st = make_tmap_3d_bf16(&ta, da, (uint64_t)kpad, (uint64_t)M, (uint64_t)n, kTK, kTM);
    if (st != ALP_OK) return st;
    st = make_tmap_3d_bf16(&tb, db, (uint64_t)kpad, (uint64_t)N, (uint64_t)n, kTK, kTN / 2);
    if (st != ALP_OK) return st;
    EmulGemmParams p;
    p.M = M;
    p.N = N;
    p.K = K;
    p.s = n;
    p.digit_bits = kDigitBits;
    p.trim = 0;
    p.crt = 1;
    for (int l = 0; l < kCrtMaxModuli; ++l) p.crt_y[l] = l < n ? crt_weight(n, l) : 0;
    p.G = reinterpret_cast<int32_t*>(G);
    p.ldg = ldg;
    p.gplane = M * ldg;
    const int64_t tiles_m = (M + kTM - 1) / kTM, tiles_n = (N + kTN - 1) / kTN;
    const int64_t pair_tiles = ((tiles_m + 1) / 2) * tiles_n;
    if (pair_tiles * 16 > 0x7fffffff) return ALP_ERR_UNSUPPORTED;
    p.tiles_m = (int)tiles_m;
    p.tiles_n = (int)tiles_n;
    p.group_m = group_m > 0 ? group_m : emul_group_m(true);
    p.timeout_ns = wait_timeout_ns();
    p.err = device_error_word();
    p.inject_skip_it = inject_skip_kt();
    cudaError_t ce = cudaFuncSetAttribute(emul_crt_fused_pair_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          kFusedSmemBytes);
    if (ce != cudaSuccess) return cuda_status(ce);
    const int P = fused_active_clusters() < kMaxFusedClusters ? fused_active_clusters()
                                                               : kMaxFusedClusters;
    p.n_full = (int)pair_tiles;
    p.pieces = 1;
    p.t_ranges = (uint64_t)(n - 1) << 4;
    if (emul_tail_split_on()) {   // whole tiles fill the waves of P clusters
        const TailSplit ts = tail_split((int)pair_tiles, n, P, false, true);
        p.n_full = ts.n_full;
        p.pieces = ts.pieces;
        p.t_ranges = 0;
        for (int i = 0; i < ts.pieces; ++i)
            p.t_ranges |= (uint64_t)((ts.t_lo[i] - 2) | (ts.t_hi[i] - 2) << 4) << (8 * i);
    }
    const int64_t items = p.n_full + (pair_tiles - p.n_full) * p.pieces;
    CrtFuse fz;
    fz.e = e;
    fz.f = f;
    fz.alpha = alpha;
    fz.beta = beta;
    fz.C = C;
    fz.ldc = ldc;
    fz.amode = alpha == 1.0 ? 0 : alpha == -1.0 ? 1 : 2;
    fz.bmode = beta != 0.0 ? 1 : 0;
    fz.n_items = (int)items;
    fz.sched = sched;
    fz.stride = (int)items + 1;
    fz.cc = crt_rec_consts(n, k);
    const int64_t clusters = items < P ? items : P;
    // the counter and every cluster's list start at all ones (-1: not yet taken)
    ce = cudaMemsetAsync(sched, 0xff, (size_t)4 * (1 + (size_t)clusters * fz.stride), stream);
    if (ce != cudaSuccess) return cuda_status(ce);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(2 * clusters));
    lc.blockDim = dim3(kFusedThreads);
    lc.dynamicSmemBytes = kFusedSmemBytes;
    lc.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    ce = cudaLaunchKernelEx(&lc, emul_crt_fused_pair_kernel, ta, tb, p, fz);
    if (ce != cudaSuccess) return cuda_status(ce);
    if (p.n_full < pair_tiles) {
        crt_tail_recombine_kernel<<<(unsigned)((pair_tiles - p.n_full) * 16), 256, 0, stream>>>(
            p, fz);
        ce = cudaGetLastError();
    }
    return cuda_status(ce);
}

}  // namespace alp
