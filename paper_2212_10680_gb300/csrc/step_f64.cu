// Kernel instantiations for storage precision ST_F64.
#include "fmlbm_launch.cuh"

namespace fmlbm {
FMLBM_DEFINE_LAUNCHERS(ST_F64)
// the FP64 path (the parity reference) has no TMA variant
template <>
cudaError_t launch_step_tma<ST_F64>(const StepArgs&, int, const CUtensorMap*, int, bool, cudaStream_t) {
    return cudaErrorNotSupported;
}
template <>
bool tma_supported<ST_F64>(int) { return false; }
// nor a paired step (it packs float arithmetic)
template <>
cudaError_t launch_step_pair<ST_F64>(const StepArgs&, int, cudaStream_t) {
    return cudaErrorNotSupported;
}
template <>
bool pair_supported<ST_F64>(int) { return false; }
}  // namespace fmlbm
