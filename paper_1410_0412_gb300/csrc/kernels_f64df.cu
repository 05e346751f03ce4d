// Instantiates the step kernels for IEEE double storage with double-float arithmetic.
#include "kernels.cuh"

namespace lbm {
LBM_INSTANTIATE_STEP_LAUNCHERS(LBM_F64_DF)
}  // namespace lbm
