// Entry points whose kernels are not in this build yet.
#include "alp_internal.cuh"

extern "C" {

alp_status alp_gemm_batched_varsize(int64_t, const int64_t*, const int64_t*, const int64_t*,
                                    const double*, const double* const*, const int64_t*,
                                    const double* const*, const int64_t*, const double*,
                                    double* const*, const int64_t*, const int64_t*,
                                    const int64_t*, const int64_t*, void*, size_t, void*) {
    return ALP_ERR_UNSUPPORTED;
}
size_t alp_gemm_batched_workspace(int64_t, const int64_t*, const int64_t*, const int64_t*) {
    return 0;
}
alp_status alp_tune(int64_t, int64_t, int64_t, alp_path, alp_tune_mode, alp_config*, double*) {
    return ALP_ERR_UNSUPPORTED;
}
}
