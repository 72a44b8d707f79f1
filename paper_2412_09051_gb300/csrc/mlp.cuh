// Learned collision correction (not part of the paper's method): a Q -> 64 ->
// 64 -> Q tanh MLP maps the non-equilibrium moments of the streamed
// populations to a correction of the post-collision f, projected so that mass,
// momentum and energy are unchanged.
//
//   z_k = sum_i Phi_ki f^neq_i             Phi: weighted-orthonormal moment basis
//   x = s_in (.) z
//   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), o = W3 h2 + b3
//   delta f_i = w_i sigma (P o)_i           P: weighted-orthogonal projection
//                                           off {1, xi, |xi|^2}
// Weights are BF16 (held as BF16-exact floats in shared memory), activations
// and accumulation FP32.
#pragma once
#include "sllbm_internal.h"

namespace sllbm {

constexpr int MLP_H = 64;

// shared-memory / global image of the network, floats:
// W1[H][Q] | W2[H][H] | W3[Q][H] | b1[H] | b2[H] | b3[Q] | s_in[Q] | Phi[Q][Q] | Ginv[(D+2)^2] | sigma
__host__ __device__ constexpr int mlp_image_floats(int Q, int D) {
    return MLP_H * Q + MLP_H * MLP_H + Q * MLP_H + 2 * MLP_H + Q + Q + Q * Q + (D + 2) * (D + 2) + 1;
}

// floats of the three weight matrices at the head of the image
__host__ __device__ constexpr int mlp_weight_floats(int Q) { return MLP_H * Q + MLP_H * MLP_H + Q * MLP_H; }

template <int Q, int D>
struct MlpView {
    const float* W1;
    const float* W2;
    const float* W3;
    const float* b1;
    const float* b2;
    const float* b3;
    const float* s_in;
    const float* phi;
    const float* ginv;
    float sigma;
    __device__ __forceinline__ explicit MlpView(const float* s) {
        W1 = s;
        W2 = W1 + MLP_H * Q;
        W3 = W2 + MLP_H * MLP_H;
        b1 = W3 + Q * MLP_H;
        b2 = b1 + MLP_H;
        b3 = b2 + MLP_H;
        s_in = b3 + Q;
        phi = s_in + Q;
        ginv = phi + Q * Q;
        sigma = ginv[(D + 2) * (D + 2)];
    }
    // view of the image's tail only (biases onward): the tensor-core path keeps
    // the weights as BF16 operand tiles instead
    struct TailOnly {};
    __device__ __forceinline__ MlpView(const float* tail, TailOnly) {
        W1 = W2 = W3 = nullptr;
        b1 = tail;
        b2 = b1 + MLP_H;
        b3 = b2 + MLP_H;
        s_in = b3 + Q;
        phi = s_in + Q;
        ginv = phi + Q * Q;
        sigma = ginv[(D + 2) * (D + 2)];
    }
};

// copy the image from global to shared memory (whole block)
template <int Q, int D>
__device__ __forceinline__ void mlp_load(const float* __restrict__ g, float* s) {
    constexpr int n = mlp_image_floats(Q, D);
    for (int k = threadIdx.x; k < n; k += blockDim.x) s[k] = __ldg(g + k);
    __syncthreads();
}

// non-equilibrium moments z (Q) from f^neq
template <int Q, int D, typename real>
__device__ __forceinline__ void mlp_moments(const MlpView<Q, D>& M, const real (&fneq)[Q], float (&z)[Q]) {
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        float a = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) a += M.phi[k * Q + i] * float(fneq[i]);
        z[k] = a;
    }
}

template <int Q, int D, typename real>
__device__ __forceinline__ void mlp_project_add(const MlpView<Q, D>& M, const CollideConst<real>& C,
                                                const float (&o)[Q], real (&f)[Q]);

// correction of the post-collision f (deviation storage: adds delta f)
template <int Q, int D, typename real>
__device__ __forceinline__ void mlp_correct(const MlpView<Q, D>& M, const CollideConst<real>& C, const float (&z)[Q],
                                            real (&f)[Q]) {
    float x[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) x[k] = M.s_in[k] * z[k];
    float h1[MLP_H];
#pragma unroll 4
    for (int j = 0; j < MLP_H; ++j) {
        float a = M.b1[j];
#pragma unroll
        for (int k = 0; k < Q; ++k) a += M.W1[j * Q + k] * x[k];
        h1[j] = tanhf(a);
    }
    float o[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) o[i] = M.b3[i];
#pragma unroll 2
    for (int j = 0; j < MLP_H; ++j) {
        float a = M.b2[j];
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) a += M.W2[j * MLP_H + k] * h1[k];
        const float h = tanhf(a);
#pragma unroll
        for (int i = 0; i < Q; ++i) o[i] += M.W3[i * MLP_H + j] * h;
    }
    mlp_project_add<Q, D, real>(M, C, o, f);
}

// f += w_i sigma (P o)_i: removes from o its weighted moments along
// {1, xi, |xi|^2} (inverse Gram matrix), so mass, momentum and energy are unchanged
template <int Q, int D, typename real>
__device__ __forceinline__ void mlp_project_add(const MlpView<Q, D>& M, const CollideConst<real>& C,
                                                const float (&o)[Q], real (&f)[Q]) {
    float m[D + 2];
#pragma unroll
    for (int l = 0; l < D + 2; ++l) m[l] = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float wo = float(C.w[i]) * o[i];
        float s2 = 0.f;
        m[0] += wo;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            m[1 + d] += float(C.xi[i][d]) * wo;
            s2 += float(C.xi[i][d]) * float(C.xi[i][d]);
        }
        m[D + 1] += s2 * wo;
    }
    float a[D + 2];
#pragma unroll
    for (int k = 0; k < D + 2; ++k) {
        float t = 0.f;
#pragma unroll
        for (int l = 0; l < D + 2; ++l) t += M.ginv[k * (D + 2) + l] * m[l];
        a[k] = t;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float s2 = 0.f, c = a[0];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            c += float(C.xi[i][d]) * a[1 + d];
            s2 += float(C.xi[i][d]) * float(C.xi[i][d]);
        }
        c += s2 * a[D + 1];
        f[i] += real(float(C.w[i]) * M.sigma * (o[i] - c));
    }
}

}  // namespace sllbm
