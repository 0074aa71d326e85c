// Autotuner: enumeration of the valid tile configs, CUDA-event timing of each
// on the GPU, the tuned-config cache consulted by alp_gemm_f64(cfg = NULL),
// and the append-only JSONL timing database.
//
// The paper tunes its tile size T by sweeping powers of two at one matrix
// size (N = 10240, control N = 7168) and keeping the best (Sect. 3 "Parameter
// Tuning", Fig. 3, Table 4).  Here the sweep covers the block tile, the K
// step and the per-thread tile, for any (M, N, K).
#include <cstdio>
#include <cstdlib>
#include <ctime>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "alp_ext.h"
#include "alp_internal.cuh"
#include "native_cfg.h"

namespace alp {

alp_status native_launch(const alp_config& cfg, bool use_tma, int64_t M, int64_t N, int64_t K,
                         double alpha, const double* A, int64_t lda, const double* B,
                         int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t stream,
                         int inject_skip_kt);
int native_occupancy(const alp_config& cfg, bool use_tma);
bool default_config(alp_path path, alp_config* out);
bool model_predict(int64_t M, int64_t N, int64_t K, alp_path path, alp_config* out,
                   double* pred_tflops);

namespace {
std::mutex g_tmu;
std::map<std::tuple<int64_t, int64_t, int64_t, int>, alp_config> g_cache;

const int kBM[3] = {64, 128, 256};
const int kBK[3] = {16, 32, 64};
const int kT[3] = {2, 4, 8};

std::vector<alp_config> native_configs() {
    std::vector<alp_config> v;
    for (int bm : kBM)
        for (int bn : kBM)
            for (int bk : kBK)
                for (int tm : kT)
                    for (int tn : kT)
                        if (native_config_valid(bm, bn, bk, tm, tn, 0))
                            v.push_back(alp_config{bm, bn, bk, tm, tn, 0});
    return v;
}
}  // namespace

std::vector<alp_config> configs_of(alp_path path) {
    if (path == ALP_PATH_NATIVE) return native_configs();
    return {};
}

bool select_config(int64_t M, int64_t N, int64_t K, alp_path path, alp_config* out) {
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        auto it = g_cache.find(std::make_tuple(M, N, K, (int)path));
        if (it != g_cache.end()) {
            *out = it->second;
            return true;
        }
    }
    if (model_predict(M, N, K, path, out, nullptr)) return true;
    return default_config(path, out);
}

void cache_config(int64_t M, int64_t N, int64_t K, alp_path path, const alp_config& c) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_cache[std::make_tuple(M, N, K, (int)path)] = c;
}

}  // namespace alp

using namespace alp;

extern "C" {

int alp_config_count(alp_path path) { return (int)configs_of(path).size(); }

alp_status alp_config_at(alp_path path, int idx, alp_config* out) {
    if (!out) return ALP_ERR_INVALID_ARG;
    auto v = configs_of(path);
    if (idx < 0 || idx >= (int)v.size()) return ALP_ERR_INVALID_ARG;
    *out = v[idx];
    return ALP_OK;
}

}  // extern "C"
