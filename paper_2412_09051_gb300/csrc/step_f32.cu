// FP32 instantiations of the fused step kernels.
#include "step_kernels.cuh"
namespace sllbm {
SLLBM_INSTANTIATE_STEP(0, 2, float)
SLLBM_INSTANTIATE_STEP(1, 2, float)
SLLBM_INSTANTIATE_STEP(1, 3, float)
SLLBM_INSTANTIATE_STEP(2, 2, float)
SLLBM_INSTANTIATE_TILED(0, float)
SLLBM_INSTANTIATE_TILED(1, float)
SLLBM_INSTANTIATE_TILED(2, float)
SLLBM_INSTANTIATE_TILED_MLP(1, float)
SLLBM_INSTANTIATE_ROW(1, float)
}  // namespace sllbm
