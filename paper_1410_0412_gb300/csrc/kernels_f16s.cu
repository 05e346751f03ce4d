// Instantiates the device kernels and launchers for LBM_F16S storage.
#include "kernels.cuh"

namespace lbm {
LBM_INSTANTIATE_LAUNCHERS(LBM_F16S)
}  // namespace lbm
