#pragma once
// Bulk asynchronous copies from global to shared memory (the TMA engine's
// untensored form, PTX cp.async.bulk) that complete on an mbarrier, and the
// mbarrier arrivals that announce them (mbarrier.arrive / .expect_tx).  The
// barrier helpers themselves (init, bounded parity wait) are in mlp_tc.cuh.
#include <cstdint>

namespace sllbm {

// arrive once on the barrier and add `bytes` to the transaction count the
// current phase waits for
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// arrive once on the barrier (a phase with no copies)
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// `bytes` (a multiple of 16) from global src to shared dst, both 16-byte
// aligned; the completed bytes count against bar's transaction count
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

}  // namespace sllbm
