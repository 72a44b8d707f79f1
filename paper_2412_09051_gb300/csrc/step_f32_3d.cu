// FP32 instantiations of the fused step kernels, 3D velocity set.
#include "step_kernels.cuh"
namespace sllbm {
SLLBM_INSTANTIATE_STEP(3, 2, float)
SLLBM_INSTANTIATE_TILED(3, float)
SLLBM_INSTANTIATE_ROW(3, float)
}  // namespace sllbm
