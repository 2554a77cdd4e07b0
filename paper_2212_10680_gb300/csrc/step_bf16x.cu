// Kernel instantiations for storage precision ST_BF16DEV_X (BF16 deviation storage with the fugacity terms of ln f in double).
// Plain step and moments only: no bulk-copy or paired form.
#include "fmlbm_launch.cuh"

namespace fmlbm {
FMLBM_DEFINE_LAUNCHERS(ST_BF16DEV_X)
template <>
cudaError_t launch_step_tma<ST_BF16DEV_X>(const StepArgs&, int, const CUtensorMap*, int, bool, cudaStream_t) {
    return cudaErrorNotSupported;
}
template <>
bool tma_supported<ST_BF16DEV_X>(int) { return false; }
template <>
cudaError_t launch_step_pair<ST_BF16DEV_X>(const StepArgs&, int, cudaStream_t) {
    return cudaErrorNotSupported;
}
template <>
bool pair_supported<ST_BF16DEV_X>(int) { return false; }
}  // namespace fmlbm
