// Kernel instantiations for storage precision ST_F16DEV.
#include "fmlbm_launch.cuh"

namespace fmlbm {
FMLBM_DEFINE_LAUNCHERS(ST_F16DEV)
FMLBM_DEFINE_TMA_LAUNCHER(ST_F16DEV)
FMLBM_DEFINE_PAIR_LAUNCHER(ST_F16DEV)
FMLBM_DEFINE_MULTI_LAUNCHER(ST_F16DEV)
}  // namespace fmlbm
