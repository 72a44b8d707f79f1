// Learned-collision MLP on the 5th-generation tensor cores (tcgen05): one CTA
// of 128 threads evaluates the network for its 128 nodes as three
// M = 128 products, one node per TMEM lane.
//
//   layer 1: D1[128 x 64]  = X [128 x K1] . W1^T      (TMEM columns 0..63)
//   layer 2: D2[128 x 64]  = H1[128 x 64] . W2^T      (TMEM columns 64..127)
//   layer 3: D3[128 x N3]  = H2[128 x 64] . W3^T      (TMEM columns 0..N3-1)
//
// Operands are BF16 in shared memory in the canonical K-major layout without
// swizzle: 8 x 16-byte core matrices, 128 B apart along K (leading byte
// offset) and K * 16 B apart along M / N (stride byte offset).  The weights
// are BF16 already; each FP32 activation x is split as x_hi = bf16(x),
// x_lo = bf16(x - x_hi) and both halves are multiplied into the same FP32
// accumulator, so the products see the activation to ~2^-17 relative and the
// network keeps its definition (BF16 weights, FP32 activations and
// accumulation) and the CUDA-core path's results to FP32 rounding.
//
// One elected thread issues the MMAs and commits them to an mbarrier; every
// wait on it is bounded (about a second of SM clock), after which the block
// records SLLBM_DEV_TC_TIMEOUT in the context's status word, skips the rest of
// the network and still frees its TMEM.
#pragma once
#include <cuda_bf16.h>
#include "mlp.cuh"

namespace sllbm {

constexpr int TC_M = 128;                 // nodes per CTA = TMEM lanes
constexpr int TC_TMEM_COLS = 128;         // D1 | D2 (D3 reuses D1's columns)

template <int Q, int D>
struct MlpTc {
    static constexpr int K1 = (Q + 15) / 16 * 16;          // layer-1 K: features, zero padded
    static constexpr int N3 = (Q + 15) / 16 * 16;          // layer-3 N: outputs, zero padded
    static constexpr int KA = K1 > MLP_H ? K1 : MLP_H;     // widest activation operand
    static constexpr int B1 = MLP_H * K1 * 2;              // bytes of each weight tile
    static constexpr int B2 = MLP_H * MLP_H * 2;
    static constexpr int B3 = N3 * MLP_H * 2;
    static constexpr int B_BYTES = B1 + B2 + B3;
    static constexpr int A_BYTES = TC_M * KA * 2;          // one of x_hi / x_lo
    static constexpr int TAIL = 2 * MLP_H + Q + Q + Q * Q + (D + 2) * (D + 2) + 1;  // floats after the weights
    static constexpr int OFF_AHI = 0;
    static constexpr int OFF_ALO = OFF_AHI + A_BYTES;
    static constexpr int OFF_B = OFF_ALO + A_BYTES;
    static constexpr int OFF_TAIL = OFF_B + B_BYTES;
    static constexpr int OFF_BAR = (OFF_TAIL + 4 * TAIL + 15) / 16 * 16;
    static constexpr int OFF_SLOT = OFF_BAR + 8;
    static constexpr int SMEM = OFF_SLOT + 8;
    static_assert(K1 % 16 == 0 && N3 % 16 == 0 && N3 >= 16 && N3 <= 256, "MMA shape");
    static_assert(MLP_H + MLP_H <= TC_TMEM_COLS && N3 <= MLP_H, "TMEM columns");
};

// byte offset of element (r, k) of an R x K BF16 operand in the canonical
// K-major no-swizzle layout (K a multiple of 8)
__host__ __device__ constexpr int tc_canon_offset(int r, int k, int K) {
    return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// non-blocking test of the phase with the given parity
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with the given parity: false after `limit` SM
// cycles (default 2^31, about a second).  A shorter (test) limit polls
// without blocking: try_wait may suspend the thread for longer than the
// limit, which would hide a short one.
constexpr long long kWaitLimit = 1ll << 31;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = kWaitLimit) {
    // a phase already complete under the default bound needs no clock read
    if (limit >= kWaitLimit && mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    if (limit < kWaitLimit) {
        while (!mbar_test(bar, parity))
            if (clock64() - t0 > limit) return false;
        return true;
    }
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
// the wait limit of the kernels that take the context's status words: word 1
// holds log2 of a test limit (sllbm_debug_wait_limit), 0 for the default
__device__ __forceinline__ long long wait_limit(const int* status) {
    const int e = status ? __ldg(status + 1) : 0;
    return e > 0 && e < 62 ? (1ll << e) : kWaitLimit;
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp-collective;
// the wait is in the same statement, so the values are complete on return)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 h) {
    return uint32_t(__bfloat16_as_ushort(h.x)) | (uint32_t(__bfloat16_as_ushort(h.y)) << 16);
}

// writes 8 activations (columns 8c .. 8c+7 of row r of an R x K operand) as
// their BF16 hi and lo parts
template <int K>
__device__ __forceinline__ void tc_put8(unsigned char* Ahi, unsigned char* Alo, int r, int c, const float* v) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
        const float2 hf = __bfloat1622float2(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
        h[e] = bf16x2_bits(hh);
        l[e] = bf16x2_bits(ll);
    }
    const int off = tc_canon_offset(r, 8 * c, K);
    *reinterpret_cast<uint4*>(Ahi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(Alo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Block-wide set-up (all 128 threads, before any of them may leave): the
// image's tail (biases, input scales, moment basis, inverse Gram matrix,
// sigma) and the BF16 weight tiles into shared memory, TMEM allocation by
// warp 0, the MMA barrier.  Returns the TMEM base address.
template <int Q, int D>
__device__ __forceinline__ uint32_t mlp_tc_setup(const float* __restrict__ img, const uint16_t* __restrict__ wimg,
                                                 unsigned char* sm) {
    using L = MlpTc<Q, D>;
    float* tail = reinterpret_cast<float*>(sm + L::OFF_TAIL);
    for (int k = threadIdx.x; k < L::TAIL; k += blockDim.x) tail[k] = __ldg(img + mlp_weight_floats(Q) + k);
    const uint4* src = reinterpret_cast<const uint4*>(wimg);
    uint4* dst = reinterpret_cast<uint4*>(sm + L::OFF_B);
    for (int k = threadIdx.x; k < L::B_BYTES / 16; k += blockDim.x) dst[k] = __ldg(src + k);
    if (threadIdx.x < 32) {
        tc_alloc(smem_u32(sm + L::OFF_SLOT), TC_TMEM_COLS);
        tc_relinquish();
    }
    if (threadIdx.x == 0) mbar_init(smem_u32(sm + L::OFF_BAR), 1);
    fence_async_smem();   // weight tiles written by the generic proxy, read by the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *reinterpret_cast<volatile uint32_t*>(sm + L::OFF_SLOT);
}

// one layer: D = [A_hi | A_lo] . [B | B]^T over K, issued by thread 0; every
// thread waits for the commit.  Returns false (block-uniform) if the wait ran out.
template <int K, int N>
__device__ __forceinline__ bool tc_layer(uint32_t ahi, uint32_t alo, uint32_t b, uint32_t d, uint32_t bar,
                                         uint32_t parity, long long limit) {
    fence_async_smem();   // this thread's activation rows -> async proxy
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_fence_after();
        constexpr uint32_t id = tc_idesc_bf16(TC_M, N);
#pragma unroll
        for (int kk = 0; kk < K / 16; ++kk) {
            const uint64_t bd = tc_sdesc(b + kk * 256, 128, K * 16);
            tc_mma(d, tc_sdesc(ahi + kk * 256, 128, K * 16), bd, id, kk > 0 ? 1u : 0u);
            tc_mma(d, tc_sdesc(alo + kk * 256, 128, K * 16), bd, id, 1u);
        }
        tc_commit(bar);
    }
    const bool ok = mbar_wait(bar, parity, limit);
    // a wait that ran out: wait once more, with the default bound, for the
    // products still in flight before the caller reuses their operands or
    // frees the tensor memory they write (the block still reports the timeout)
    if (!ok) mbar_wait(bar, parity);
    tc_fence_after();
    return __syncthreads_and(ok) != 0;
}

// Correction of the post-collision f of this thread's node by the network on
// the tensor cores (whole block; z: the node's non-equilibrium moments, zero
// on threads that carry no node).  Frees the block's TMEM on return.
template <int Q, int D, typename real>
__device__ __forceinline__ void mlp_correct_tc(const MlpView<Q, D>& M, const CollideConst<real>& C, unsigned char* sm,
                                               uint32_t tbase, const float (&z)[Q], real (&f)[Q],
                                               int* __restrict__ status) {
    using L = MlpTc<Q, D>;
    unsigned char* Ahi = sm + L::OFF_AHI;
    unsigned char* Alo = sm + L::OFF_ALO;
    const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo), bar = smem_u32(sm + L::OFF_BAR);
    const uint32_t bw1 = smem_u32(sm + L::OFF_B), bw2 = bw1 + L::B1, bw3 = bw2 + L::B2;
    const int r = threadIdx.x;
    const uint32_t trow = tbase + (uint32_t(r & ~31) << 16);   // this warp's 32 TMEM lanes

    // layer-1 operand: scaled features, zero beyond Q
#pragma unroll
    for (int c = 0; c < L::K1 / 8; ++c) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = 8 * c + e;
            v[e] = k < Q ? M.s_in[k < Q ? k : 0] * z[k < Q ? k : 0] : 0.f;
        }
        tc_put8<L::K1>(Ahi, Alo, r, c, v);
    }
    const long long lim = wait_limit(status);
    bool ok = tc_layer<L::K1, MLP_H>(ahi, alo, bw1, tbase, bar, 0, lim);
    if (ok) {
#pragma unroll 1   // runtime chunk loops keep the tanh code small (instruction fetch)
        for (int c = 0; c < MLP_H / 16; ++c) {
            float v[16];
            tc_ld16(trow + 16 * c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = tanhf(v[j] + M.b1[16 * c + j]);
            tc_put8<MLP_H>(Ahi, Alo, r, 2 * c, v);
            tc_put8<MLP_H>(Ahi, Alo, r, 2 * c + 1, v + 8);
        }
        ok = tc_layer<MLP_H, MLP_H>(ahi, alo, bw2, tbase + MLP_H, bar, 1, lim);
    }
    if (ok) {
#pragma unroll 1
        for (int c = 0; c < MLP_H / 16; ++c) {
            float v[16];
            tc_ld16(trow + MLP_H + 16 * c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = tanhf(v[j] + M.b2[16 * c + j]);
            tc_put8<MLP_H>(Ahi, Alo, r, 2 * c, v);
            tc_put8<MLP_H>(Ahi, Alo, r, 2 * c + 1, v + 8);
        }
        ok = tc_layer<MLP_H, L::N3>(ahi, alo, bw3, tbase, bar, 0, lim);
    }
    if (ok) {
        float o[Q];
#pragma unroll
        for (int c = 0; c < L::N3 / 16; ++c) {
            float v[16];
            tc_ld16(trow + 16 * c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (16 * c + j < Q) o[16 * c + j] = v[j] + M.b3[16 * c + j];
        }
        mlp_project_add<Q, D, real>(M, C, o, f);
    } else if (r == 0) {
        atomicOr(status, SLLBM_DEV_TC_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (r < 32) {
        tc_fence_after();
        tc_dealloc(tbase, TC_TMEM_COLS);
    }
}

}  // namespace sllbm
