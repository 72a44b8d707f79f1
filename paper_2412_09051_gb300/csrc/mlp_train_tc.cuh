// Training of the learned collision correction on the 5th-generation tensor
// cores (tcgen05): forward and backward pass of one 128-sample tile per CTA
// (one sample per thread and per tensor-memory lane), BF16 operands and FP32
// accumulation in tensor memory.  The network is the one mlp_tc.cuh
// evaluates: BF16 weights, FP32 activations (each activation or delta split
// into BF16 hi and lo parts, both multiplied into the accumulator), so the
// gradients match the CUDA-core trainer's (k_train_batch) to FP32 rounding.
//
//   forward   D1 = X . W1^T,  h1 = tanh(D1 + b1)          (M 128, N 64, K K1)
//             D2 = H1 . W2^T, h2 = tanh(D2 + b2)          (M 128, N 64, K 64)
//             D3 = H2 . W3^T, o = D3 + b3                 (M 128, N N3, K 64)
//   loss      r = P (o - y), L += sum w r^2, g = scale P^T (w r)   (CUDA cores)
//   backward  d2 = (G . W3) (1 - h2^2)                    (M 128, N 64, K K1)
//             d1 = (D2 . W2) (1 - h1^2)                   (M 128, N 64, K 64)
//   gradients over the samples (K = 128), three products per K step
//             (hi hi + hi lo + lo hi):
//             [H1^T; H2^T] . [D2^T; G^T]^T -> dW2^T (rows 0-63, columns
//             0-63), dW3^T (rows 64-127, columns 64 ..)
//             [X^T; ...; 1] . [D1^T; D2^T; G^T]^T -> dW1^T (rows < Q,
//             columns 0-63) and, from the row of ones, db1 | db2 | db3
//
// Each CTA adds its tile's gradients to the global sums with one atomic per
// parameter.  Every wait on the MMA barrier is bounded (mlp_tc.cuh): a block
// whose wait runs out records it in the trainer's status word, stops, and
// still frees its tensor memory.
#pragma once
#include <cuda_bf16.h>

#include "mlp_tc.cuh"

namespace sllbm {

template <int Q>
struct TrainTc {
    static constexpr int H = MLP_H;
    static constexpr int K1 = (Q + 15) / 16 * 16;     // input features / outputs, zero padded
    static constexpr int N3 = K1;
    static constexpr int S = 128;                     // samples per CTA
    static constexpr int GBR = 2 * H + N3;            // rows of the gradient B operand: D1^T | D2^T | G^T
    // weight tiles (BF16, K-major canonical)
    static constexpr int OFF_W1 = 0;                  // [H x K1]: (j, q) = W1[j][q]
    static constexpr int OFF_W2 = OFF_W1 + H * K1 * 2;        // [H x H]: (j, q) = W2[j][q]
    static constexpr int OFF_W3 = OFF_W2 + H * H * 2;         // [N3 x H]: (i, j) = W3[i][j]
    static constexpr int OFF_W3B = OFF_W3 + N3 * H * 2;       // [H x K1]: (j, i) = W3[i][j]
    static constexpr int OFF_W2B = OFF_W3B + H * K1 * 2;      // [H x H]: (q, j) = W2[j][q]
    // activation operands: the layer operand [128 x <= 64] hi / lo aliases the
    // first 16 KB of the gradient A operand [128 x 128] hi / lo
    static constexpr int OFF_GAH = OFF_W2B + H * H * 2;
    static constexpr int OFF_GAL = OFF_GAH + S * S * 2;
    static constexpr int OFF_GBH = OFF_GAL + S * S * 2;
    static constexpr int OFF_GBL = OFF_GBH + GBR * S * 2;
    static constexpr int OFF_F = OFF_GBL + GBR * S * 2;       // floats: P [Q][Q], w, b1, b2, b3
    static constexpr int NF = Q * Q + Q + H + H + Q;
    static constexpr int OFF_BAR = (OFF_F + 4 * NF + 15) / 16 * 16;
    static constexpr int OFF_SLOT = OFF_BAR + 8;
    static constexpr int OFF_RED = OFF_SLOT + 8;             // 4 warp partial losses
    static constexpr int SMEM = OFF_RED + 16;
    static constexpr int TMEM_COLS = 512;                     // D regions 0..255, h1 256..319, h2 320..383
    static constexpr int C_H1 = 256, C_H2 = 320;
    static_assert(K1 <= H && GBR <= 256 && H + N3 <= 256, "MMA shapes");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// 16 FP32 values into columns [taddr, taddr + 16) of this thread's lane
__device__ __forceinline__ void tr_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tr_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// one element of an R x K operand at (r, k), as its BF16 hi and lo parts
template <int K>
__device__ __forceinline__ void tr_put1(unsigned char* Ahi, unsigned char* Alo, int r, int k, float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    const int off = tc_canon_offset(r, k, K);
    *reinterpret_cast<__nv_bfloat16*>(Ahi + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(Alo + off) = l;
}

// D[128 x N] = A . B^T over K with A and B both split: A_hi B_hi + A_hi B_lo
// + A_lo B_hi per K step of 16, issued by thread 0; every thread waits for
// the commit.  B may start at any multiple of 8 rows of its buffer (bhi, blo
// point there).  Returns false (block-uniform) if the wait ran out.
template <int K, int N>
__device__ __forceinline__ bool tr_layer3(uint32_t ahi, uint32_t alo, uint32_t bhi, uint32_t blo, uint32_t d,
                                          uint32_t bar, uint32_t parity, long long limit) {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_fence_after();
        constexpr uint32_t id = tc_idesc_bf16(TC_M, N);
#pragma unroll
        for (int kk = 0; kk < K / 16; ++kk) {
            const uint64_t ah = tc_sdesc(ahi + kk * 256, 128, K * 16), al = tc_sdesc(alo + kk * 256, 128, K * 16);
            const uint64_t bh = tc_sdesc(bhi + kk * 256, 128, K * 16), bl = tc_sdesc(blo + kk * 256, 128, K * 16);
            tc_mma(d, ah, bh, id, kk > 0 ? 1u : 0u);
            tc_mma(d, ah, bl, id, 1u);
            tc_mma(d, al, bh, id, 1u);
        }
        tc_commit(bar);
    }
    const bool ok = mbar_wait(bar, parity, limit);
    if (!ok) mbar_wait(bar, parity);
    tc_fence_after();
    return __syncthreads_and(ok) != 0;
}


// One 128-sample tile of the batch per CTA (128 threads); gradients and the
// loss are added to B.grad and B.loss.  TrainBufs and POff come from the
// including file (mlp_train.cu).
template <int Q>
__global__ void __launch_bounds__(128, 1)
    k_train_tc(const TrainBufs B, int64_t off, int count, float scale, int* __restrict__ status) {
    using L = TrainTc<Q>;
    using O = POff<Q>;
    constexpr int H = L::H, K1 = L::K1, N3 = L::N3;
    extern __shared__ __align__(128) float sm_f[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(sm_f);
    const int t = threadIdx.x;     // sample t of the tile, tensor-memory lane t
    float* F = reinterpret_cast<float*>(sm + L::OFF_F);
    float* Pm = F;
    float* wv = Pm + Q * Q;
    float* b1 = wv + Q;
    float* b2 = b1 + H;
    float* b3 = b2 + H;
    auto bf = [&](int offset) { return reinterpret_cast<__nv_bfloat16*>(sm + offset); };
    // weight tiles (the parameters are BF16-rounded already: exact), the
    // projector, the weights w_i and the biases
    for (int e = t; e < H * K1; e += 128) {
        const int j = e / K1, q = e % K1;
        *bf(L::OFF_W1 + tc_canon_offset(j, q, K1)) = __float2bfloat16_rn(q < Q ? B.pr[O::W1 + j * Q + q] : 0.f);
        *bf(L::OFF_W3B + tc_canon_offset(j, q, K1)) = __float2bfloat16_rn(q < Q ? B.pr[O::W3 + q * H + j] : 0.f);
    }
    for (int e = t; e < H * H; e += 128) {
        const int j = e / H, q = e % H;
        const __nv_bfloat16 v = __float2bfloat16_rn(B.pr[O::W2 + j * H + q]);
        *bf(L::OFF_W2 + tc_canon_offset(j, q, H)) = v;
        *bf(L::OFF_W2B + tc_canon_offset(q, j, H)) = v;
    }
    for (int e = t; e < N3 * H; e += 128) {
        const int i = e / H, j = e % H;
        *bf(L::OFF_W3 + tc_canon_offset(i, j, H)) = __float2bfloat16_rn(i < Q ? B.pr[O::W3 + i * H + j] : 0.f);
    }
    for (int e = t; e < Q * Q; e += 128) Pm[e] = B.P[e];
    for (int e = t; e < Q; e += 128) {
        wv[e] = B.w[e];
        b3[e] = B.pr[O::b3 + e];
    }
    for (int e = t; e < H; e += 128) {
        b1[e] = B.pr[O::b1 + e];
        b2[e] = B.pr[O::b2 + e];
    }
    if (t < 32) {
        tc_alloc(smem_u32(sm + L::OFF_SLOT), L::TMEM_COLS);
        tc_relinquish();
    }
    if (t == 0) mbar_init(smem_u32(sm + L::OFF_BAR), 1);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(sm + L::OFF_SLOT);
    const uint32_t trow = tbase + (uint32_t(t & ~31) << 16);
    unsigned char* Ahi = sm + L::OFF_GAH;
    unsigned char* Alo = sm + L::OFF_GAL;
    unsigned char* Bhi = sm + L::OFF_GBH;
    unsigned char* Blo = sm + L::OFF_GBL;
    const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo), bhi = smem_u32(Bhi), blo = smem_u32(Blo);
    const uint32_t bar = smem_u32(sm + L::OFF_BAR);
    const long long lim = wait_limit(status);
    const int64_t s0 = off + int64_t(blockIdx.x) * L::S;
    const int ns = int(min(int64_t(L::S), off + count - s0));
    const bool real = t < ns;
    const int64_t srow = s0 + t;
    uint32_t ph = 0;
    float lsum = 0.f;

    // ---- forward
#pragma unroll
    for (int c = 0; c < K1 / 8; ++c) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int q = 8 * c + e;
            v[e] = (real && q < Q) ? B.X[srow * Q + q] : 0.f;
        }
        tc_put8<K1>(Ahi, Alo, t, c, v);
    }
    bool ok = tc_layer<K1, H>(ahi, alo, smem_u32(sm + L::OFF_W1), tbase, bar, ph, lim);
    ph ^= 1;
    if (ok) {
#pragma unroll 1
        for (int c = 0; c < H / 16; ++c) {
            float v[16];
            tc_ld16(trow + 16 * c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = tanhf(v[j] + b1[16 * c + j]);
            tr_st16(trow + L::C_H1 + 16 * c, v);
            tc_put8<H>(Ahi, Alo, t, 2 * c, v);
            tc_put8<H>(Ahi, Alo, t, 2 * c + 1, v + 8);
        }
        ok = tc_layer<H, H>(ahi, alo, smem_u32(sm + L::OFF_W2), tbase + 64, bar, ph, lim);
        ph ^= 1;
    }
    if (ok) {
#pragma unroll 1
        for (int c = 0; c < H / 16; ++c) {
            float v[16];
            tc_ld16(trow + 64 + 16 * c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = tanhf(v[j] + b2[16 * c + j]);
            tr_st16(trow + L::C_H2 + 16 * c, v);
            tc_put8<H>(Ahi, Alo, t, 2 * c, v);
            tc_put8<H>(Ahi, Alo, t, 2 * c + 1, v + 8);
        }
        ok = tc_layer<H, N3>(ahi, alo, smem_u32(sm + L::OFF_W3), tbase, bar, ph, lim);
        ph ^= 1;
    }
    // ---- loss and dL/do (CUDA cores): r = P (o - y), L += sum w r^2, g = scale P^T (w r)
    if (ok) {
        float e[K1], r[Q];
#pragma unroll
        for (int c = 0; c < N3 / 16; ++c) {
            float v[16];
            tc_ld16(trow + 16 * c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int i = 16 * c + j;
                e[i] = (real && i < Q) ? v[j] + b3[i < Q ? i : 0] - B.Y[srow * Q + (i < Q ? i : 0)] : 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float a = 0.f;
#pragma unroll
            for (int j = 0; j < Q; ++j) a += Pm[i * Q + j] * e[j];
            lsum += wv[i] * a * a;
            r[i] = wv[i] * a;
        }
#pragma unroll
        for (int i = 0; i < K1; ++i) {
            float a = 0.f;
            if (i < Q) {
#pragma unroll
                for (int j = 0; j < Q; ++j) a += Pm[j * Q + i] * r[j];
            }
            e[i] = scale * a;       // g
        }
        // G: A operand of the d2 product; G^T: rows 2H .. of the gradient B operand
#pragma unroll
        for (int c = 0; c < K1 / 8; ++c) tc_put8<K1>(Ahi, Alo, t, c, e + 8 * c);
#pragma unroll
        for (int i = 0; i < N3; ++i) tr_put1<L::S>(Bhi, Blo, 2 * H + i, t, e[i]);
        tr_wait_st();       // h1, h2 in tensor memory before they are read back
        ok = tc_layer<K1, H>(ahi, alo, smem_u32(sm + L::OFF_W3B), tbase + 128, bar, ph, lim);
        ph ^= 1;
    }
    // ---- backward: d2 = (G . W3) (1 - h2^2)
    if (ok) {
#pragma unroll 1
        for (int c = 0; c < H / 16; ++c) {
            float v[16], h[16];
            tc_ld16(trow + 128 + 16 * c, v);
            tc_ld16(trow + L::C_H2 + 16 * c, h);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] *= 1.f - h[j] * h[j];
            tc_put8<H>(Ahi, Alo, t, 2 * c, v);
            tc_put8<H>(Ahi, Alo, t, 2 * c + 1, v + 8);
#pragma unroll
            for (int j = 0; j < 16; ++j) tr_put1<L::S>(Bhi, Blo, H + 16 * c + j, t, v[j]);
        }
        ok = tc_layer<H, H>(ahi, alo, smem_u32(sm + L::OFF_W2B), tbase + 192, bar, ph, lim);
        ph ^= 1;
    }
    // d1 = (D2 . W2) (1 - h1^2) -> rows 0 .. H-1 of the gradient B operand;
    // the gradient A operand [H1^T; H2^T] overwrites the layer operand (its
    // last product has completed)
    if (ok) {
#pragma unroll 1
        for (int c = 0; c < H / 16; ++c) {
            float v[16], h[16];
            tc_ld16(trow + 192 + 16 * c, v);
            tc_ld16(trow + L::C_H1 + 16 * c, h);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                tr_put1<L::S>(Bhi, Blo, 16 * c + j, t, v[j] * (1.f - h[j] * h[j]));
                tr_put1<L::S>(Ahi, Alo, 16 * c + j, t, h[j]);
            }
            tc_ld16(trow + L::C_H2 + 16 * c, h);
#pragma unroll
            for (int j = 0; j < 16; ++j) tr_put1<L::S>(Ahi, Alo, H + 16 * c + j, t, h[j]);
        }
        // [H1^T; H2^T] . [D2^T; G^T]^T: B from row H of its buffer
        constexpr uint32_t brow = uint32_t(H / 8) * uint32_t(L::S * 16);
        ok = tr_layer3<L::S, H + N3>(ahi, alo, bhi + brow, blo + brow, tbase, bar, ph, lim);
        ph ^= 1;
    }
    if (ok) {
        if (t < H) {          // warps 0, 1: row q = t: dW2[j][q] in columns 0 .. H-1
#pragma unroll 1
            for (int c = 0; c < H / 16; ++c) {
                float v[16];
                tc_ld16(trow + 16 * c, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) atomicAdd(B.grad + O::W2 + (16 * c + j) * H + t, v[j]);
            }
        } else {              // warps 2, 3: row H + j: dW3[i][j] in columns H + i
#pragma unroll 1
            for (int c = 0; c < N3 / 16; ++c) {
                float v[16];
                tc_ld16(trow + H + 16 * c, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int i = 16 * c + j;
                    if (i < Q) atomicAdd(B.grad + O::W3 + i * H + (t - H), v[j]);
                }
            }
        }
        // gradient A operand [X^T; ...; ones]: rows 0 .. K1-1 the inputs, row
        // 127 ones (the bias sums); rows between keep finite values whose
        // products are not read
#pragma unroll 1
        for (int q = 0; q < K1; ++q) tr_put1<L::S>(Ahi, Alo, q, t, (real && q < Q) ? B.X[srow * Q + q] : 0.f);
        tr_put1<L::S>(Ahi, Alo, L::S - 1, t, 1.f);
        ok = tr_layer3<L::S, L::GBR>(ahi, alo, bhi, blo, tbase, bar, ph, lim);
        ph ^= 1;
    }
    if (ok) {
        const int w = t >> 5;
        if (w * 32 < K1) {    // rows q < K1: dW1[j][q] in columns 0 .. H-1
#pragma unroll 1
            for (int c = 0; c < H / 16; ++c) {
                float v[16];
                tc_ld16(trow + 16 * c, v);
                if (t < Q) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) atomicAdd(B.grad + O::W1 + (16 * c + j) * Q + t, v[j]);
                }
            }
        }
        if (w == 3) {         // row 127: db1 | db2 | db3
#pragma unroll 1
            for (int c = 0; c < L::GBR / 16; ++c) {
                float v[16];
                tc_ld16(trow + 16 * c, v);
                if (t == L::S - 1) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int k = 16 * c + j;
                        if (k < H)
                            atomicAdd(B.grad + O::b1 + k, v[j]);
                        else if (k < 2 * H)
                            atomicAdd(B.grad + O::b2 + (k - H), v[j]);
                        else if (k - 2 * H < Q)
                            atomicAdd(B.grad + O::b3 + (k - 2 * H), v[j]);
                    }
                }
            }
        }
    }
    // ---- the tile's loss; a wait that ran out is recorded
    float* red = reinterpret_cast<float*>(sm + L::OFF_RED);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((t & 31) == 0) red[t >> 5] = lsum;
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
        atomicAdd(B.loss, red[0] + red[1] + red[2] + red[3]);
        if (!ok) atomicOr(status, SLLBM_DEV_TC_TIMEOUT);
    }
    if (t < 32) {
        tc_fence_after();
        tc_dealloc(tbase, L::TMEM_COLS);
    }
}

}  // namespace sllbm
