// Cost model (placeholder until the MLP kernels land).
#include "alp_internal.cuh"

namespace alp {
bool model_predict(int64_t, int64_t, int64_t, alp_path, alp_config*, double*) { return false; }
}  // namespace alp
