// Kernel instantiations for storage precision ST_F64.
#include "fmlbm_launch.cuh"

namespace fmlbm {
FMLBM_DEFINE_LAUNCHERS(ST_F64)
}  // namespace fmlbm
