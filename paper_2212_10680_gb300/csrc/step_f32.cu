// Kernel instantiations for storage precision ST_F32.
#include "fmlbm_launch.cuh"

namespace fmlbm {
FMLBM_DEFINE_LAUNCHERS(ST_F32)
FMLBM_DEFINE_TMA_LAUNCHER(ST_F32)
FMLBM_DEFINE_PAIR_LAUNCHER(ST_F32)
FMLBM_DEFINE_MULTI_LAUNCHER(ST_F32)
}  // namespace fmlbm
