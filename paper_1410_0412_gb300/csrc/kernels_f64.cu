// Instantiates the device kernels and launchers for LBM_F64 storage.
#include "kernels.cuh"

namespace lbm {
LBM_INSTANTIATE_LAUNCHERS(LBM_F64)
}  // namespace lbm
