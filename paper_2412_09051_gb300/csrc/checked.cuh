#pragma once
// Bounds checks of the debug build.  Compiled with -DSLLBM_CHECKED, every index
// that a step kernel reads from a record table or derives from one (the
// record slot, the source population, the boundary-state id, the source node
// along each axis or relative to the arriving node, the cell of a gather code,
// the slot of a shared-memory row buffer) passes through SLLBM_CHK: an index
// outside [0, n) sets a bit of the context's device status word
// (SLLBM_DEV_BAD_*, read by sllbm_device_status) and is replaced by 0, which is
// inside every buffer, so a bad record shows up as a status bit and a wrong
// result instead of a memory fault.  Nothing traps or waits.  Without the
// macro SLLBM_CHK expands to its index alone: the release kernels are
// unchanged, and the status pointer is never read.
#include "sllbm.h"

namespace sllbm {

#ifdef SLLBM_CHECKED
template <typename I, typename J>
__device__ __forceinline__ I chk_index(I idx, J n, int* status, int bit) {
    if (idx >= 0 && idx < n) return idx;
    if (status) atomicOr(status, bit);
    return I(0);
}
#define SLLBM_CHK(idx, n, status, bit) (::sllbm::chk_index((idx), (n), (status), (bit)))
// a load offset rel relative to the arriving node n: n + rel must lie in [0, N)
#define SLLBM_CHK_REL(n, rel, N, status) \
    (::sllbm::chk_index((n) + (rel), (N), (status), SLLBM_DEV_BAD_NODE) - (n))
#else
#define SLLBM_CHK(idx, n, status, bit) (idx)
#define SLLBM_CHK_REL(n, rel, N, status) (rel)
#endif

}  // namespace sllbm
