// Batched variable-size native FP64 GEMM: thousands of independent problems
// C_p = alpha_p A_p B_p + beta_p C_p in one persistent launch.
//
// 1. A one-block plan kernel classifies every problem by its tile class
//    (row and column tile of 32, 64 or 128, from M and N), orders problems by
//    class and then by K bucket, longest first, and writes the prefix sum of
//    their tile counts: the device work list.  Everything it reads is device
//    memory, so the call is stream-ordered and capturable in a CUDA graph.
// 2. A persistent kernel (one block of 8 warps per SM) takes tiles from an
//    atomic counter, finds each tile's problem by binary search in the prefix
//    array, and runs the tile with the register tile of its class
//    (tm = bm/16, tn = bn/16, the native kernel's DMMA building blocks, loads
//    through cp.async since every problem has its own pointers).
//
// The class -> (bm, bn, bk) table is runtime state (alp_batched_set_class_config)
// so that an autotuner can set it per class.
#include <cstdlib>
#include <mutex>

#include "alp_ext.h"
#include "native.cuh"

namespace alp {

namespace {

constexpr int kClasses = 9;           // 3 row-tile x 3 column-tile sizes
constexpr int kKBuckets = 16;         // floor(log2 K) buckets, longest first
constexpr int kBatchedThreads = 256;  // 8 warps: (bm/(8 tm)) x (bn/(4 tn)) with tm = bm/16, tn = bn/16
constexpr int kPlanThreads = 1024;

struct ClassTable {
    int bm[kClasses], bn[kClasses], bk[kClasses];
};

std::mutex g_bmu;
ClassTable g_table = {
    {32, 32, 32, 64, 64, 64, 128, 128, 128},
    {32, 64, 128, 32, 64, 128, 32, 64, 128},
    {32, 32, 16, 32, 16, 16, 16, 16, 16}};

ClassTable current_table() {
    std::lock_guard<std::mutex> lk(g_bmu);
    return g_table;
}

__host__ __device__ __forceinline__ int size_bucket(int64_t v) { return v <= 32 ? 0 : v <= 64 ? 1 : 2; }
__host__ __device__ __forceinline__ int class_of(int64_t M, int64_t N) {
    return size_bucket(M) * 3 + size_bucket(N);
}

struct BatchArgs {
    int64_t count;
    const int64_t *M, *N, *K, *lda, *ldb, *ldc;
    const double *alpha, *beta;
    const double* const* A;
    const double* const* B;
    double* const* C;
};

struct Plan {              // device workspace
    int32_t* key;          // [count] sort key per problem (-1: nothing to do)
    int32_t* order;        // [count] problem ids in (class, K bucket desc) order
    int64_t* prefix;       // [count + 1] exclusive tile prefix over `order`
    int64_t* meta;         // [0] valid problems, [1] total tiles
    unsigned long long* counter;   // tile counter of the persistent kernel
};

__global__ void __launch_bounds__(kPlanThreads) batched_plan_kernel(BatchArgs a, Plan pl,
                                                                   ClassTable tab) {
    __shared__ int cnt[kClasses * kKBuckets];
    __shared__ int base[kClasses * kKBuckets];
    __shared__ int64_t chunk_sum[kPlanThreads];
    __shared__ int64_t carry;
    const int tid = threadIdx.x;
    for (int i = tid; i < kClasses * kKBuckets; i += kPlanThreads) cnt[i] = 0;
    __syncthreads();
    for (int64_t p = tid; p < a.count; p += kPlanThreads) {
        const int64_t M = a.M[p], N = a.N[p];
        int64_t K = a.K[p];
        if (a.alpha[p] == 0.0) K = 0;
        int key = -1;
        if (M > 0 && N > 0) {
            const int kb = K > 0 ? 63 - __clzll((long long)K) : 0;
            key = class_of(M, N) * kKBuckets + (kKBuckets - 1 - (kb < kKBuckets ? kb : kKBuckets - 1));
            atomicAdd(&cnt[key], 1);
        }
        pl.key[p] = key;
    }
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int i = 0; i < kClasses * kKBuckets; ++i) {
            base[i] = run;
            run += cnt[i];
        }
        pl.meta[0] = run;
    }
    __syncthreads();
    for (int64_t p = tid; p < a.count; p += kPlanThreads) {
        const int key = pl.key[p];
        if (key >= 0) pl.order[atomicAdd(&base[key], 1)] = (int32_t)p;
    }
    __syncthreads();
    // exclusive prefix of tile counts along `order`, 1024 entries at a time
    const int64_t nvalid = pl.meta[0];
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nvalid; c0 += kPlanThreads) {
        const int64_t pos = c0 + tid;
        int64_t tiles = 0;
        if (pos < nvalid) {
            const int32_t p = pl.order[pos];
            const int c = class_of(a.M[p], a.N[p]);
            tiles = ((a.M[p] + tab.bm[c] - 1) / tab.bm[c]) * ((a.N[p] + tab.bn[c] - 1) / tab.bn[c]);
        }
        chunk_sum[tid] = tiles;
        __syncthreads();
        for (int off = 1; off < kPlanThreads; off <<= 1) {   // inclusive Hillis-Steele scan
            const int64_t v = tid >= off ? chunk_sum[tid - off] : 0;
            __syncthreads();
            chunk_sum[tid] += v;
            __syncthreads();
        }
        if (pos < nvalid) pl.prefix[pos] = carry + chunk_sum[tid] - tiles;
        __syncthreads();
        if (tid == kPlanThreads - 1) carry += chunk_sum[tid];
        __syncthreads();
    }
    if (tid == 0) {
        pl.prefix[nvalid] = carry;
        pl.meta[1] = carry;
        *pl.counter = 0ull;
    }
}

template <int TM, int TN>
__device__ __forceinline__ void run_tile(const TileProblem& pr, int64_t m0, int64_t n0, int bm, int bn,
                                         int bk, double* smem, bool vec2) {
    tile_ldg<TM, TN>(pr, m0, n0, bm, bn, bk, smem, vec2);
}

// MAXT: the largest bm and bn the class table may hold.  With MAXT = 64 only
// the register tiles up to 4 x 4 are compiled, which fit two blocks per SM;
// with MAXT = 32 only 2 x 2, three blocks per SM.
template <int MAXT>
__global__ void __launch_bounds__(kBatchedThreads, MAXT <= 32 ? 3 : MAXT <= 64 ? 2 : 1)
    batched_persistent_kernel(BatchArgs a, Plan pl, ClassTable tab) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int64_t s_tile;
    double* smem = reinterpret_cast<double*>(smem_raw);
    const int64_t total = pl.meta[1];
    const int64_t nvalid = pl.meta[0];
    while (true) {
        if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(pl.counter, 1ull);
        __syncthreads();
        const int64_t t = s_tile;
        __syncthreads();
        if (t >= total) break;
        // position: last pos with prefix[pos] <= t
        int64_t lo = 0, hi = nvalid - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (pl.prefix[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const int32_t p = pl.order[lo];
        const int64_t local = t - pl.prefix[lo];
        TileProblem pr;
        pr.M = a.M[p];
        pr.N = a.N[p];
        pr.alpha = a.alpha[p];
        pr.beta = a.beta[p];
        pr.K = pr.alpha == 0.0 ? 0 : a.K[p];
        pr.A = a.A[p];
        pr.B = a.B[p];
        pr.C = a.C[p];
        pr.lda = a.lda[p];
        pr.ldb = a.ldb[p];
        pr.ldc = a.ldc[p];
        const int c = class_of(pr.M, pr.N);
        const int bm = tab.bm[c], bn = tab.bn[c], bk = tab.bk[c];
        const int64_t tiles_n = (pr.N + bn - 1) / bn;
        const int64_t m0 = (local / tiles_n) * bm, n0 = (local % tiles_n) * bn;
        const bool vec2 = ((reinterpret_cast<uintptr_t>(pr.C) & 15) == 0) && (pr.ldc % 2 == 0);
        const int tm = bm / 16, tn = bn / 16;
#define ALP_BATCHED_CASE(x, y) \
    if (tm == x && tn == y) run_tile<x, y>(pr, m0, n0, bm, bn, bk, smem, vec2);
        if (MAXT <= 32) {
            ALP_BATCHED_CASE(2, 2)
        } else if (MAXT <= 64) {
            ALP_BATCHED_CASE(2, 2) else ALP_BATCHED_CASE(2, 4) else ALP_BATCHED_CASE(4, 2)
            else ALP_BATCHED_CASE(4, 4)
        } else {
            ALP_BATCHED_CASE(2, 2) else ALP_BATCHED_CASE(2, 4) else ALP_BATCHED_CASE(2, 8)
            else ALP_BATCHED_CASE(4, 2) else ALP_BATCHED_CASE(4, 4) else ALP_BATCHED_CASE(4, 8)
            else ALP_BATCHED_CASE(8, 2) else ALP_BATCHED_CASE(8, 4) else ALP_BATCHED_CASE(8, 8)
        }
#undef ALP_BATCHED_CASE
    }
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct PlanLayout {
    size_t off_key, off_order, off_prefix, off_meta, off_counter, bytes;
};

PlanLayout plan_layout(int64_t count) {
    PlanLayout L;
    size_t off = 0;
    L.off_key = off; off += up256((size_t)count * 4);
    L.off_order = off; off += up256((size_t)count * 4);
    L.off_prefix = off; off += up256((size_t)(count + 1) * 8);
    L.off_meta = off; off += 256;
    L.off_counter = off; off += 256;
    L.bytes = off;
    return L;
}

// Largest bm or bn among the classes in `present` (bit c: class c has tiles).
int max_tile(const ClassTable& t, unsigned present) {
    int m = 0;
    for (int c = 0; c < kClasses; ++c) {
        if (!(present >> c & 1u)) continue;
        m = t.bm[c] > m ? t.bm[c] : m;
        m = t.bn[c] > m ? t.bn[c] : m;
    }
    return m;
}

int max_smem(const ClassTable& t) {
    int m = 0;
    for (int c = 0; c < kClasses; ++c) {
        const int b = 2 * (t.bm[c] + t.bn[c]) * t.bk[c] * 8;
        m = b > m ? b : m;
    }
    return m;
}

// The persistent kernel for `tiles` tiles on `sms` SMs, as many blocks as fit.
// When the classes present use tiles of at most 64 x 64 (32 x 32) it runs the
// variant that fits two (three) blocks per SM.
alp_status launch_persistent(const BatchArgs& a, const Plan& pl, const ClassTable& tab,
                             int64_t tiles, unsigned present, int sms, cudaStream_t stream) {
    const int smem = max_smem(tab);
    const int mt = max_tile(tab, present);
    auto kernel = mt <= 32   ? batched_persistent_kernel<32>
                  : mt <= 64 ? batched_persistent_kernel<64>
                             : batched_persistent_kernel<128>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_status(e);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kBatchedThreads, smem);
    if (occ < 1) occ = 1;
    int64_t grid = (int64_t)sms * occ;
    if (grid > tiles) grid = tiles;
    kernel<<<(unsigned)grid, kBatchedThreads, smem, stream>>>(a, pl, tab);
    return cuda_status(cudaGetLastError());
}

}  // namespace

// Launches plan + persistent kernel for the whole batch on `sms` SMs, with the
// work list in `workspace` (256-byte aligned, plan_layout(count).bytes).
alp_status batched_launch(const BatchArgs& a, const int64_t* hM, const int64_t* hN,
                          void* workspace, cudaStream_t stream, int sms) {
    const ClassTable tab = current_table();
    const PlanLayout L = plan_layout(a.count);
    char* ws = static_cast<char*>(workspace);
    Plan pl;
    pl.key = reinterpret_cast<int32_t*>(ws + L.off_key);
    pl.order = reinterpret_cast<int32_t*>(ws + L.off_order);
    pl.prefix = reinterpret_cast<int64_t*>(ws + L.off_prefix);
    pl.meta = reinterpret_cast<int64_t*>(ws + L.off_meta);
    pl.counter = reinterpret_cast<unsigned long long*>(ws + L.off_counter);
    // grid size from the host copies (performance only: the persistent loop
    // covers any number of tiles)
    int64_t tiles = 0;
    unsigned present = 0;
    for (int64_t p = 0; p < a.count; ++p) {
        if (hM[p] <= 0 || hN[p] <= 0) continue;
        const int c = class_of(hM[p], hN[p]);
        tiles += ((hM[p] + tab.bm[c] - 1) / tab.bm[c]) * ((hN[p] + tab.bn[c] - 1) / tab.bn[c]);
        present |= 1u << c;
    }
    batched_plan_kernel<<<1, kPlanThreads, 0, stream>>>(a, pl, tab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    if (tiles == 0) return ALP_OK;
    return launch_persistent(a, pl, tab, tiles, present, sms, stream);
}

}  // namespace alp

using namespace alp;

namespace {
bool class_config_ok(int bm, int bn, int bk) {
    auto ok = [](int v) { return v == 32 || v == 64 || v == 128; };
    return ok(bm) && ok(bn) && (bk == 16 || bk == 32 || bk == 64) &&
           2 * (bm + bn) * bk * 8 <= kSmemLimit;
}

alp_status fill_args(BatchArgs& a, int64_t count, const int64_t* dM, const int64_t* dN,
                     const int64_t* dK, const double* dalpha, const double* const* dA,
                     const int64_t* dlda, const double* const* dB, const int64_t* dldb,
                     const double* dbeta, double* const* dC, const int64_t* dldc) {
    if (!dM || !dN || !dK || !dalpha || !dA || !dlda || !dB || !dldb || !dbeta || !dC || !dldc)
        return ALP_ERR_INVALID_ARG;
    a.count = count;
    a.M = dM; a.N = dN; a.K = dK; a.alpha = dalpha; a.beta = dbeta;
    a.A = dA; a.B = dB; a.C = dC; a.lda = dlda; a.ldb = dldb; a.ldc = dldc;
    return ALP_OK;
}

alp_status check_host_sizes(int64_t count, const int64_t* hM, const int64_t* hN,
                            const int64_t* hK) {
    if (count < 0 || count > 0x7fffffff) return ALP_ERR_INVALID_ARG;
    if (count > 0 && (!hM || !hN || !hK)) return ALP_ERR_INVALID_ARG;
    for (int64_t p = 0; p < count; ++p)
        if (hM[p] < 0 || hN[p] < 0 || hK[p] < 0) return ALP_ERR_INVALID_ARG;
    return ALP_OK;
}

struct BatchedGraph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};
}  // namespace

extern "C" {

size_t alp_gemm_batched_workspace(int64_t count, const int64_t* hM, const int64_t* hN,
                                  const int64_t* hK) {
    if (check_host_sizes(count, hM, hN, hK) != ALP_OK) return 0;
    return plan_layout(count).bytes;
}

alp_status alp_gemm_batched_varsize(int64_t count, const int64_t* dM, const int64_t* dN,
                                    const int64_t* dK, const double* dalpha,
                                    const double* const* dA, const int64_t* dlda,
                                    const double* const* dB, const int64_t* dldb,
                                    const double* dbeta, double* const* dC,
                                    const int64_t* dldc, const int64_t* hM,
                                    const int64_t* hN, const int64_t* hK, void* workspace,
                                    size_t workspace_bytes, void* stream) {
    alp_status st = check_host_sizes(count, hM, hN, hK);
    if (st != ALP_OK) return st;
    if (count == 0) return ALP_OK;
    BatchArgs a;
    if ((st = fill_args(a, count, dM, dN, dK, dalpha, dA, dlda, dB, dldb, dbeta, dC, dldc)) !=
        ALP_OK)
        return st;
    if (!workspace || workspace_bytes < plan_layout(count).bytes || ((uintptr_t)workspace & 255))
        return ALP_ERR_WORKSPACE;
    return batched_launch(a, hM, hN, workspace, reinterpret_cast<cudaStream_t>(stream),
                          device_sm_count());
}

alp_status alp_batched_set_class_config(int cls, int bm, int bn, int bk) {
    if (cls < 0 || cls >= kClasses || !class_config_ok(bm, bn, bk)) return ALP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_bmu);
    g_table.bm[cls] = bm;
    g_table.bn[cls] = bn;
    g_table.bk[cls] = bk;
    return ALP_OK;
}

alp_status alp_batched_get_class_config(int cls, int* bm, int* bn, int* bk) {
    if (cls < 0 || cls >= kClasses || !bm || !bn || !bk) return ALP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_bmu);
    *bm = g_table.bm[cls];
    *bn = g_table.bn[cls];
    *bk = g_table.bk[cls];
    return ALP_OK;
}

int alp_batched_class_of(int64_t M, int64_t N) { return class_of(M, N); }

alp_status alp_batched_graph_create(int64_t count, const int64_t* dM, const int64_t* dN,
                                    const int64_t* dK, const double* dalpha,
                                    const double* const* dA, const int64_t* dlda,
                                    const double* const* dB, const int64_t* dldb,
                                    const double* dbeta, double* const* dC,
                                    const int64_t* dldc, const int64_t* hM,
                                    const int64_t* hN, const int64_t* hK, void* workspace,
                                    size_t workspace_bytes, void** graph_out) {
    if (!graph_out) return ALP_ERR_INVALID_ARG;
    *graph_out = nullptr;
    // one-time per-device set-up (error word, SM count) must not happen
    // inside the capture
    if (!device_error_word() || device_sm_count() < 1) return ALP_ERR_CUDA;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return ALP_ERR_CUDA;
    BatchedGraph* g = new BatchedGraph{nullptr, nullptr};
    alp_status st = ALP_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        st = ALP_ERR_CUDA;
    } else {
        st = alp_gemm_batched_varsize(count, dM, dN, dK, dalpha, dA, dlda, dB, dldb, dbeta, dC,
                                      dldc, hM, hN, hK, workspace, workspace_bytes, cs);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (st == ALP_OK && e != cudaSuccess) st = ALP_ERR_CUDA;
        g->graph = graph;
        if (st == ALP_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess)
            st = ALP_ERR_CUDA;
    }
    cudaStreamDestroy(cs);
    if (st != ALP_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return st;
    }
    *graph_out = g;
    return ALP_OK;
}

alp_status alp_batched_graph_launch(void* graph, void* stream) {
    if (!graph) return ALP_ERR_INVALID_ARG;
    BatchedGraph* g = static_cast<BatchedGraph*>(graph);
    return cuda_status(cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)));
}

alp_status alp_batched_graph_destroy(void* graph) {
    if (!graph) return ALP_OK;
    BatchedGraph* g = static_cast<BatchedGraph*>(graph);
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return ALP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched GEMM without a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they issue
// the GEMM: frameworks whose device memory is owned by their own pool
// allocator, and real-time or long-running loops that must not take the
// allocator's locks or risk the implicit device synchronisation of
// cudaMalloc / cudaFree.  For them this entry point keeps the work list of
// the persistent kernel in one file-scope device array instead of a
// workspace.  The array is part of the library image: every GPU that loads
// the library holds these kNoAllocScratchBytes until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;   // 1 MiB: up to 65,000 problems
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64];   // device address of g_noalloc_scratch per device (nullptr: not set up)
int g_noalloc_sms[64];     // SM count per device

// Device address of the scratch array on the current device and its SM count.
// The first call on a device looks both up (cudaGetSymbolAddress and an
// attribute query, neither of which allocates); later calls reuse them.
alp_status noalloc_scratch(void** out, int* sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ALP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ALP_ERR_CUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            n < 1)
            return ALP_ERR_CUDA;
        g_noalloc_sms[dev] = n;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    *sms = g_noalloc_sms[dev];
    return ALP_OK;
}
}  // namespace

extern "C" alp_status alp_gemm_batched_varsize_noalloc(
    int64_t count, const int64_t* dM, const int64_t* dN, const int64_t* dK, const double* dalpha,
    const double* const* dA, const int64_t* dlda, const double* const* dB, const int64_t* dldb,
    const double* dbeta, double* const* dC, const int64_t* dldc, const int64_t* hM,
    const int64_t* hN, const int64_t* hK, void* stream) {
    alp_status st = check_host_sizes(count, hM, hN, hK);
    if (st != ALP_OK) return st;
    if (count == 0) return ALP_OK;
    if (plan_layout(count).bytes > kNoAllocScratchBytes) return ALP_ERR_WORKSPACE;   // too many problems
    BatchArgs a;
    if ((st = fill_args(a, count, dM, dN, dK, dalpha, dA, dlda, dB, dldb, dbeta, dC, dldc)) !=
        ALP_OK)
        return st;
    void* scratch = nullptr;
    int sms = 0;
    if ((st = noalloc_scratch(&scratch, &sms)) != ALP_OK) return st;
    // The same launch as alp_gemm_batched_varsize with the scratch array as its
    // workspace (256-byte aligned, as a workspace must be).  The plan kernel
    // rewrites every part of it that it later reads (keys, order, prefix sums,
    // counts, and the tile counter it sets to 0), so the previous call's
    // contents need no clearing.
    return batched_launch(a, hM, hN, scratch, reinterpret_cast<cudaStream_t>(stream), sms);
}
