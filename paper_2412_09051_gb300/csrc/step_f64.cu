// FP64 instantiations of the fused step kernels.
#include "step_kernels.cuh"
namespace sllbm {
SLLBM_INSTANTIATE_STEP(0, 2, double)
SLLBM_INSTANTIATE_STEP(1, 2, double)
SLLBM_INSTANTIATE_STEP(1, 3, double)
SLLBM_INSTANTIATE_STEP(2, 2, double)
SLLBM_INSTANTIATE_STEP(3, 2, double)
SLLBM_INSTANTIATE_TILED(0, double)
SLLBM_INSTANTIATE_TILED(1, double)
SLLBM_INSTANTIATE_TILED(2, double)
SLLBM_INSTANTIATE_TILED(3, double)
}  // namespace sllbm
