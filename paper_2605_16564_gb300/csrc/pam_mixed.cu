// pam_mixed.cu -- the mixed-precision form (tensor-core Gram, fp32 solve
// with iterative refinement). Not built yet: the plan rejects it.
#include "pam_internal.cuh"

namespace pam {
void launch_solve_level_mixed(const Geo &, const Par &, const int32_t *, const double *, double *,
                              int32_t *, const Ws &, cudaStream_t) {}
void launch_residual_mixed(const Geo &, const int32_t *, const double *, const double *,
                           const int32_t *, const Ws &, cudaStream_t) {}
void launch_eval_mixed(const Geo &, const int32_t *, const double *, const double *,
                       const int32_t *, const double *, int64_t, double *, int, cudaStream_t) {}
}  // namespace pam
