// FP32 instantiations of the fused step kernels for order p = 4 cells (the
// order of every case in the paper's Sec. 4): 2D sets with the unrolled
// kernels, D3Q45 (125 taps per population) with the runtime-loop ones.
#include "step_kernels.cuh"
namespace sllbm {
SLLBM_INSTANTIATE_STEP(0, 4, float)
SLLBM_INSTANTIATE_STEP(1, 4, float)
SLLBM_INSTANTIATE_STEP(2, 4, float)
SLLBM_INSTANTIATE_STEP_COMPACT(3, 4, float)
SLLBM_INSTANTIATE_TILED_P(0, 4, float)
SLLBM_INSTANTIATE_TILED_P(1, 4, float)
SLLBM_INSTANTIATE_TILED_P(2, 4, float)
SLLBM_INSTANTIATE_TILED_P(3, 4, float)
SLLBM_INSTANTIATE_ROWP(1, float)
SLLBM_INSTANTIATE_ROWP(3, float)
}  // namespace sllbm
