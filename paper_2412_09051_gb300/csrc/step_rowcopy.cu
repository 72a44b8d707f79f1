// FP32 instantiations of the one-block-per-row step kernel whose source rows
// are staged by the bulk-copy engine (2D and 3D velocity sets).
#include "step_kernels.cuh"
namespace sllbm {
SLLBM_INSTANTIATE_ROWC(1, float)
SLLBM_INSTANTIATE_ROWC(3, float)
}  // namespace sllbm
