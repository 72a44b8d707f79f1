// FP64 instantiations of the fused step kernels for order p = 4 cells.
#include "step_kernels.cuh"
namespace sllbm {
SLLBM_INSTANTIATE_STEP(0, 4, double)
SLLBM_INSTANTIATE_STEP(1, 4, double)
SLLBM_INSTANTIATE_STEP(2, 4, double)
SLLBM_INSTANTIATE_STEP_COMPACT(3, 4, double)
SLLBM_INSTANTIATE_TILED_P(0, 4, double)
SLLBM_INSTANTIATE_TILED_P(1, 4, double)
SLLBM_INSTANTIATE_TILED_P(2, 4, double)
SLLBM_INSTANTIATE_TILED_P(3, 4, double)
}  // namespace sllbm
