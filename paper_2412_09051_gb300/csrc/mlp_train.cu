// Training of the learned collision correction (not part of the paper's
// method): forward, backward and Adam update kernels in FP32 with the forward
// pass on BF16-rounded weights (the precision the step kernel runs), plus the
// host-side construction of the moment basis and the conservation projection.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "mlp.cuh"

namespace sllbm {

// ------------------------------------------------------------ host algebra
// Phi: modified Gram-Schmidt of graded monomials in <a,b> = sum w a b;
// Ginv: inverse Gram matrix of {1, xi, |xi|^2}; P = I - C^T Ginv C W.
void build_moment_basis(const HostVelSet& vs, std::vector<double>& Phi, std::vector<double>& Ginv,
                        std::vector<double>& P, std::vector<int>* degree) {
    const int Q = vs.Q, D = vs.D;
    std::vector<std::vector<double>> rows;
    if (degree) degree->clear();
    auto dot = [&](const std::vector<double>& a, const std::vector<double>& b) {
        double s = 0;
        for (int i = 0; i < Q; ++i) s += vs.w[i] * a[i] * b[i];
        return s;
    };
    for (int deg = 0; deg <= 12 && int(rows.size()) < Q; ++deg) {
        std::vector<std::array<int, 3>> mons;
        if (D == 2) {
            for (int a = deg; a >= 0; --a) mons.push_back({a, deg - a, 0});
        } else {
            for (int a = deg; a >= 0; --a)
                for (int b = deg - a; b >= 0; --b) mons.push_back({a, b, deg - a - b});
        }
        for (const auto& m : mons) {
            if (int(rows.size()) == Q) break;
            std::vector<double> v(Q);
            for (int i = 0; i < Q; ++i) {
                double t = 1;
                for (int d = 0; d < D; ++d)
                    for (int e = 0; e < m[d]; ++e) t *= vs.xi[i * D + d];
                v[i] = t;
            }
            const double n0 = std::sqrt(dot(v, v));
            for (const auto& r : rows) {
                const double c = dot(v, r);
                for (int i = 0; i < Q; ++i) v[i] -= c * r[i];
            }
            const double n = std::sqrt(dot(v, v));
            if (n > 1e-9 * std::max(n0, 1.0)) {
                for (int i = 0; i < Q; ++i) v[i] /= n;
                rows.push_back(v);
                if (degree) degree->push_back(deg);
            }
        }
    }
    Phi.assign(size_t(Q) * Q, 0.0);
    for (int k = 0; k < int(rows.size()); ++k)
        for (int i = 0; i < Q; ++i) Phi[k * Q + i] = rows[k][i];
    const int K = D + 2;
    std::vector<double> Cm(size_t(K) * Q);
    for (int i = 0; i < Q; ++i) {
        double s2 = 0;
        Cm[0 * Q + i] = 1.0;
        for (int d = 0; d < D; ++d) {
            Cm[(1 + d) * Q + i] = vs.xi[i * D + d];
            s2 += vs.xi[i * D + d] * vs.xi[i * D + d];
        }
        Cm[(D + 1) * Q + i] = s2;
    }
    std::vector<double> G(size_t(K) * K, 0.0), A(size_t(K) * 2 * K, 0.0);
    for (int k = 0; k < K; ++k)
        for (int l = 0; l < K; ++l) {
            double s = 0;
            for (int i = 0; i < Q; ++i) s += Cm[k * Q + i] * vs.w[i] * Cm[l * Q + i];
            G[k * K + l] = s;
        }
    // Gauss-Jordan inverse with partial pivoting
    for (int k = 0; k < K; ++k) {
        for (int l = 0; l < K; ++l) A[k * 2 * K + l] = G[k * K + l];
        A[k * 2 * K + K + k] = 1.0;
    }
    for (int c = 0; c < K; ++c) {
        int piv = c;
        for (int r = c + 1; r < K; ++r)
            if (std::fabs(A[r * 2 * K + c]) > std::fabs(A[piv * 2 * K + c])) piv = r;
        for (int l = 0; l < 2 * K; ++l) std::swap(A[c * 2 * K + l], A[piv * 2 * K + l]);
        const double d = A[c * 2 * K + c];
        for (int l = 0; l < 2 * K; ++l) A[c * 2 * K + l] /= d;
        for (int r = 0; r < K; ++r) {
            if (r == c) continue;
            const double f = A[r * 2 * K + c];
            for (int l = 0; l < 2 * K; ++l) A[r * 2 * K + l] -= f * A[c * 2 * K + l];
        }
    }
    Ginv.assign(size_t(K) * K, 0.0);
    for (int k = 0; k < K; ++k)
        for (int l = 0; l < K; ++l) Ginv[k * K + l] = A[k * 2 * K + K + l];
    P.assign(size_t(Q) * Q, 0.0);
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) {
            double s = i == j ? 1.0 : 0.0;
            for (int k = 0; k < K; ++k)
                for (int l = 0; l < K; ++l) s -= Cm[k * Q + i] * Ginv[k * K + l] * Cm[l * Q + j] * vs.w[j];
            P[i * Q + j] = s;
        }
}

void build_moment_basis(const HostVelSet& vs, std::vector<double>& Phi, std::vector<double>& Ginv,
                        std::vector<double>& P) {
    build_moment_basis(vs, Phi, Ginv, P, nullptr);
}

// ------------------------------------------------------------ device kernels
constexpr int TS = 32;     // samples per block
constexpr int TT = 256;    // threads per block

__host__ __device__ constexpr int n_params(int Q) { return MLP_H * Q + MLP_H + MLP_H * MLP_H + MLP_H + Q * MLP_H + Q; }

struct TrainBufs {
    int Q;
    int64_t M;
    const float* X;      // normalised inputs [M][Q]
    const float* Y;      // normalised targets [M][Q]
    const float* pr;     // BF16-rounded parameters (forward weights), biases unrounded
    float* grad;         // [n_params]
    const float* P;      // [Q][Q]
    const float* w;      // [Q]
    float* loss;         // accumulated loss
};

// parameter offsets in the flattened vector: W1 | b1 | W2 | b2 | W3 | b3
template <int Q>
struct POff {
    static constexpr int W1 = 0, b1 = MLP_H * Q, W2 = b1 + MLP_H, b2 = W2 + MLP_H * MLP_H, W3 = b2 + MLP_H,
                         b3 = W3 + Q * MLP_H, N = b3 + Q;
};

template <int Q>
__global__ void __launch_bounds__(TT) k_train_batch(const TrainBufs B, int64_t off, int count, float scale) {
    using O = POff<Q>;
    extern __shared__ float sm[];
    float* W = sm;                       // O::N
    float* P = W + O::N;                 // Q*Q
    float* w = P + Q * Q;                // Q
    float* x = w + Q;                    // TS*Q
    float* h1 = x + TS * Q;              // TS*H
    float* h2 = h1 + TS * MLP_H;         // TS*H
    float* r = h2 + TS * MLP_H;          // TS*Q (residual, then w-weighted)
    float* g = r + TS * Q;               // TS*Q  dL/do
    float* d2 = g + TS * Q;              // TS*H  dL/d(pre-activation 2)
    float* d1 = d2 + TS * MLP_H;         // TS*H
    __shared__ float red[TT / 32];
    const int t = threadIdx.x;
    for (int k = t; k < O::N; k += TT) W[k] = B.pr[k];
    for (int k = t; k < Q * Q; k += TT) P[k] = B.P[k];
    for (int k = t; k < Q; k += TT) w[k] = B.w[k];
    const int64_t s0 = off + int64_t(blockIdx.x) * TS;
    const int ns = int(min(int64_t(TS), off + count - s0));
    for (int k = t; k < TS * Q; k += TT) {
        const int s = k / Q;
        x[k] = s < ns ? B.X[(s0 + s) * Q + (k % Q)] : 0.f;
    }
    __syncthreads();
    for (int k = t; k < TS * MLP_H; k += TT) {
        const int s = k / MLP_H, j = k % MLP_H;
        float a = W[O::b1 + j];
        for (int q = 0; q < Q; ++q) a += W[O::W1 + j * Q + q] * x[s * Q + q];
        h1[k] = tanhf(a);
    }
    __syncthreads();
    for (int k = t; k < TS * MLP_H; k += TT) {
        const int s = k / MLP_H, j = k % MLP_H;
        float a = W[O::b2 + j];
        for (int q = 0; q < MLP_H; ++q) a += W[O::W2 + j * MLP_H + q] * h1[s * MLP_H + q];
        h2[k] = tanhf(a);
    }
    __syncthreads();
    // o - y into g (temporary)
    for (int k = t; k < TS * Q; k += TT) {
        const int s = k / Q, i = k % Q;
        float o = W[O::b3 + i];
        for (int j = 0; j < MLP_H; ++j) o += W[O::W3 + i * MLP_H + j] * h2[s * MLP_H + j];
        g[k] = s < ns ? o - B.Y[(s0 + s) * Q + i] : 0.f;
    }
    __syncthreads();
    // r = P (o - y); loss += sum w r^2; r <- w r
    float lsum = 0.f;
    for (int k = t; k < TS * Q; k += TT) {
        const int s = k / Q, i = k % Q;
        float a = 0.f;
        for (int j = 0; j < Q; ++j) a += P[i * Q + j] * g[s * Q + j];
        lsum += w[i] * a * a;
        r[k] = w[i] * a;
    }
    __syncthreads();
    // g = scale P^T (w r)
    for (int k = t; k < TS * Q; k += TT) {
        const int s = k / Q, i = k % Q;
        float a = 0.f;
        for (int j = 0; j < Q; ++j) a += P[j * Q + i] * r[s * Q + j];
        g[k] = scale * a;
    }
    __syncthreads();
    for (int k = t; k < TS * MLP_H; k += TT) {
        const int s = k / MLP_H, j = k % MLP_H;
        float a = 0.f;
        for (int i = 0; i < Q; ++i) a += g[s * Q + i] * W[O::W3 + i * MLP_H + j];
        const float h = h2[k];
        d2[k] = a * (1.f - h * h);
    }
    __syncthreads();
    for (int k = t; k < TS * MLP_H; k += TT) {
        const int s = k / MLP_H, q = k % MLP_H;
        float a = 0.f;
        for (int j = 0; j < MLP_H; ++j) a += d2[s * MLP_H + j] * W[O::W2 + j * MLP_H + q];
        const float h = h1[k];
        d1[k] = a * (1.f - h * h);
    }
    __syncthreads();
    // parameter gradients, summed over the block's samples
    for (int p = t; p < O::N; p += TT) {
        float a = 0.f;
        if (p < O::b1) {
            const int j = p / Q, q = p % Q;
            for (int s = 0; s < TS; ++s) a += d1[s * MLP_H + j] * x[s * Q + q];
        } else if (p < O::W2) {
            const int j = p - O::b1;
            for (int s = 0; s < TS; ++s) a += d1[s * MLP_H + j];
        } else if (p < O::b2) {
            const int j = (p - O::W2) / MLP_H, q = (p - O::W2) % MLP_H;
            for (int s = 0; s < TS; ++s) a += d2[s * MLP_H + j] * h1[s * MLP_H + q];
        } else if (p < O::W3) {
            const int j = p - O::b2;
            for (int s = 0; s < TS; ++s) a += d2[s * MLP_H + j];
        } else if (p < O::b3) {
            const int i = (p - O::W3) / MLP_H, j = (p - O::W3) % MLP_H;
            for (int s = 0; s < TS; ++s) a += g[s * Q + i] * h2[s * MLP_H + j];
        } else {
            const int i = p - O::b3;
            for (int s = 0; s < TS; ++s) a += g[s * Q + i];
        }
        atomicAdd(B.grad + p, a);
    }
    // block loss
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((t & 31) == 0) red[t >> 5] = lsum;
    __syncthreads();
    if (t == 0) {
        float s = 0.f;
        for (int k = 0; k < TT / 32; ++k) s += red[k];
        atomicAdd(B.loss, s);
    }
}

}  // namespace sllbm

#include "mlp_train_tc.cuh"

namespace sllbm {

template <int Q>
size_t train_smem() {
    return sizeof(float) * (POff<Q>::N + Q * Q + Q + TS * Q * 3 + TS * MLP_H * 4);
}

// Adam step on the master parameters; refreshes the BF16-rounded weights
// (biases are kept in FP32) and clears the gradient.
__global__ void k_adam(float* __restrict__ p, float* __restrict__ pr, float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, int n, int n_weights_mask_b1, int b1, int W2, int b2, int W3, int b3,
                       float lr, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = grad[k];
    const float mk = 0.9f * m[k] + 0.1f * gk;
    const float vk = 0.999f * v[k] + 0.001f * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + 1e-8f);
    p[k] = pk;
    const bool is_bias = (k >= b1 && k < W2) || (k >= b2 && k < W3) || (k >= b3);
    pr[k] = is_bias ? pk : __bfloat162float(__float2bfloat16_rn(pk));
    grad[k] = 0.f;
    (void)n_weights_mask_b1;
}

__global__ void k_round_params(const float* __restrict__ p, float* __restrict__ pr, int n, int b1, int W2, int b2,
                               int W3, int b3) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const bool is_bias = (k >= b1 && k < W2) || (k >= b2 && k < W3) || (k >= b3);
    pr[k] = is_bias ? p[k] : __bfloat162float(__float2bfloat16_rn(p[k]));
}

// data normalisation: per-feature mean square of z, and the weighted
// mean square of the projected targets
// target filter: R <- F R in place (F = Phi_K^T Phi_K W keeps the moments of
// the selected degrees; identity when all are kept)
__global__ void k_filter_targets(float* __restrict__ R, int64_t M, int Q, const float* __restrict__ F) {
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= M) return;
    float r[64];
    for (int j = 0; j < Q; ++j) r[j] = R[s * Q + j];
    for (int i = 0; i < Q; ++i) {
        float a = 0.f;
        for (int j = 0; j < Q; ++j) a += F[i * Q + j] * r[j];
        R[s * Q + i] = a;
    }
}

__global__ void k_data_stats(const float* __restrict__ Z, const float* __restrict__ R, int64_t M, int Q,
                             const float* __restrict__ P, const float* __restrict__ w, double* __restrict__ acc) {
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= M) return;
    for (int k = 0; k < Q; ++k) {
        const double z = Z[s * Q + k];
        atomicAdd(acc + k, z * z);
    }
    double e = 0;
    for (int i = 0; i < Q; ++i) {
        double a = 0;
        for (int j = 0; j < Q; ++j) a += double(P[i * Q + j]) * R[s * Q + j];
        e += double(w[i]) * a * a;
    }
    atomicAdd(acc + Q, e);
}

__global__ void k_normalise(const float* __restrict__ Z, const float* __restrict__ R, int64_t M, int Q,
                            const float* __restrict__ s_in, float inv_sigma, float* __restrict__ X,
                            float* __restrict__ Y) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= M * Q) return;
    X[k] = s_in[k % Q] * Z[k];
    Y[k] = inv_sigma * R[k];
}

}  // namespace sllbm

using namespace sllbm;

struct sllbm_trainer {
    int device = 0;
    int Q = 0, D = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    std::vector<double> w, Phi, Ginv, P;
    std::vector<int> degree;          // polynomial degree of each moment-basis row
    float *d_p = nullptr, *d_pr = nullptr, *d_grad = nullptr, *d_m = nullptr, *d_v = nullptr;
    float *d_P = nullptr, *d_w = nullptr, *d_loss = nullptr;
    float *d_X = nullptr, *d_Y = nullptr, *d_sin = nullptr;
    int* d_status = nullptr;           // tensor-core waits: status bits, test wait limit (log2)
    int path = SLLBM_MLP_TENSOR;       // forward / backward on the tensor cores or the CUDA cores
    int64_t M = 0;
    float sigma = 1.f;
    std::vector<float> s_in;
    int t = 0;
};

namespace {
int tfail(sllbm_trainer* t, int code, const std::string& m) {
    t->last_error = m;
    return code;
}
#define TCK(call)                                                                                       \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return tfail(tr, SLLBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <int Q>
int launch_train_tc(sllbm_trainer* tr, const TrainBufs& B, int64_t off, int count, float scale) {
    using L = TrainTc<Q>;
    if (cudaFuncSetAttribute(k_train_tc<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM) != cudaSuccess)
        return tfail(tr, SLLBM_ERR_CUDA, "cudaFuncSetAttribute failed");
    const unsigned grid = unsigned((count + L::S - 1) / L::S);
    k_train_tc<Q><<<grid, 128, L::SMEM, tr->stream>>>(B, off, count, scale, tr->d_status);
    return SLLBM_OK;
}

int launch_batch(sllbm_trainer* tr, int64_t off, int count, int batch_norm) {
    TrainBufs B{tr->Q, tr->M, tr->d_X, tr->d_Y, tr->d_pr, tr->d_grad, tr->d_P, tr->d_w, tr->d_loss};
    const unsigned grid = unsigned((count + TS - 1) / TS);
    const float scale = 2.0f / float(batch_norm);
    if (tr->path == SLLBM_MLP_TENSOR && (tr->Q == 19 || tr->Q == 45)) {
        const int rc = tr->Q == 19 ? launch_train_tc<19>(tr, B, off, count, scale)
                                   : launch_train_tc<45>(tr, B, off, count, scale);
        if (rc) return rc;
    } else if (tr->Q == 19) {
        const size_t sm = train_smem<19>();
        cudaFuncSetAttribute(k_train_batch<19>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        k_train_batch<19><<<grid, TT, sm, tr->stream>>>(B, off, count, scale);
    } else if (tr->Q == 45) {
        const size_t sm = train_smem<45>();
        cudaFuncSetAttribute(k_train_batch<45>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        k_train_batch<45><<<grid, TT, sm, tr->stream>>>(B, off, count, scale);
    } else {
        return tfail(tr, SLLBM_ERR_UNSUPPORTED, "trainer built for Q = 19 and Q = 45");
    }
    TCK(cudaGetLastError());
    return SLLBM_OK;
}

void offsets(int Q, int& b1, int& W2, int& b2, int& W3, int& b3) {
    b1 = MLP_H * Q;
    W2 = b1 + MLP_H;
    b2 = W2 + MLP_H * MLP_H;
    W3 = b2 + MLP_H;
    b3 = W3 + Q * MLP_H;
}
}  // namespace

// C ABI (declared in include/sllbm.h)
extern "C" {

int sllbm_train_create(const sllbm_ctx* ctx, const float* init_params, sllbm_trainer** out) {
    if (!ctx || !init_params || !out) return SLLBM_ERR_ARG;
    *out = nullptr;
    auto* tr = new (std::nothrow) sllbm_trainer();
    if (!tr) return SLLBM_ERR_NOMEM;
    tr->device = ctx->device;
    tr->Q = ctx->vs.Q;
    tr->D = ctx->vs.D;
    tr->stream = ctx->stream;
    cudaSetDevice(tr->device);
    build_moment_basis(ctx->vs, tr->Phi, tr->Ginv, tr->P, &tr->degree);
    tr->w = ctx->vs.w;
    const int n = n_params(tr->Q);
    auto bail = [&](int rc) {
        sllbm_train_destroy(tr);
        return rc;
    };
    float** bufs[] = {&tr->d_p, &tr->d_pr, &tr->d_grad, &tr->d_m, &tr->d_v};
    for (float** b : bufs)
        if (cudaMalloc(b, sizeof(float) * n) != cudaSuccess) return bail(SLLBM_ERR_NOMEM);
    if (cudaMalloc(&tr->d_P, sizeof(float) * tr->Q * tr->Q) != cudaSuccess) return bail(SLLBM_ERR_NOMEM);
    if (cudaMalloc(&tr->d_w, sizeof(float) * tr->Q) != cudaSuccess) return bail(SLLBM_ERR_NOMEM);
    if (cudaMalloc(&tr->d_loss, sizeof(float)) != cudaSuccess) return bail(SLLBM_ERR_NOMEM);
    if (cudaMalloc(&tr->d_sin, sizeof(float) * tr->Q) != cudaSuccess) return bail(SLLBM_ERR_NOMEM);
    if (cudaMalloc(&tr->d_status, 2 * sizeof(int)) != cudaSuccess) return bail(SLLBM_ERR_NOMEM);
    cudaMemset(tr->d_status, 0, 2 * sizeof(int));
    std::vector<float> Pf(tr->P.begin(), tr->P.end()), wf(tr->w.begin(), tr->w.end());
    cudaMemcpy(tr->d_P, Pf.data(), sizeof(float) * Pf.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(tr->d_w, wf.data(), sizeof(float) * wf.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(tr->d_p, init_params, sizeof(float) * n, cudaMemcpyHostToDevice);
    cudaMemset(tr->d_grad, 0, sizeof(float) * n);
    cudaMemset(tr->d_m, 0, sizeof(float) * n);
    cudaMemset(tr->d_v, 0, sizeof(float) * n);
    int b1, W2, b2, W3, b3;
    offsets(tr->Q, b1, W2, b2, W3, b3);
    k_round_params<<<(n + 255) / 256, 256, 0, tr->stream>>>(tr->d_p, tr->d_pr, n, b1, W2, b2, W3, b3);
    if (cudaStreamSynchronize(tr->stream) != cudaSuccess) return bail(SLLBM_ERR_CUDA);
    tr->s_in.assign(tr->Q, 1.0f);
    *out = tr;
    return SLLBM_OK;
}

int sllbm_train_destroy(sllbm_trainer* tr) {
    if (!tr) return SLLBM_OK;
    cudaSetDevice(tr->device);
    float* bufs[] = {tr->d_p, tr->d_pr, tr->d_grad, tr->d_m, tr->d_v, tr->d_P, tr->d_w, tr->d_loss,
                     tr->d_X, tr->d_Y, tr->d_sin};
    for (float* b : bufs)
        if (b) cudaFree(b);
    if (tr->d_status) cudaFree(tr->d_status);
    delete tr;
    return SLLBM_OK;
}

int sllbm_train_path(sllbm_trainer* tr, int32_t path) {
    if (!tr || (path != SLLBM_MLP_TENSOR && path != SLLBM_MLP_SIMT)) return SLLBM_ERR_ARG;
    tr->path = path;
    return SLLBM_OK;
}

const char* sllbm_train_last_error(const sllbm_trainer* tr) { return tr ? tr->last_error.c_str() : ""; }

int sllbm_train_set_data(sllbm_trainer* tr, const float* Z, const float* R, int64_t M, int32_t max_degree,
                         int32_t on_device) {
    if (!tr || !Z || !R || M <= 0 || max_degree < 0 || tr->Q > 64) return SLLBM_ERR_ARG;
    cudaSetDevice(tr->device);
    const int Q = tr->Q;
    if (tr->d_X) cudaFree(tr->d_X);
    if (tr->d_Y) cudaFree(tr->d_Y);
    tr->d_X = tr->d_Y = nullptr;
    float *dZ = nullptr, *dR = nullptr;
    double* acc = nullptr;
    TCK(cudaMalloc(&tr->d_X, sizeof(float) * M * Q));
    TCK(cudaMalloc(&tr->d_Y, sizeof(float) * M * Q));
    TCK(cudaMalloc(&dZ, sizeof(float) * M * Q));
    TCK(cudaMalloc(&dR, sizeof(float) * M * Q));
    TCK(cudaMalloc(&acc, sizeof(double) * (Q + 1)));
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    TCK(cudaMemcpyAsync(dZ, Z, sizeof(float) * M * Q, k, tr->stream));
    TCK(cudaMemcpyAsync(dR, R, sizeof(float) * M * Q, k, tr->stream));
    TCK(cudaMemsetAsync(acc, 0, sizeof(double) * (Q + 1), tr->stream));
    if (max_degree > 0) {   // keep only the target moments of degree <= max_degree
        std::vector<float> F(size_t(Q) * Q, 0.0f);
        for (int i = 0; i < Q; ++i)
            for (int j = 0; j < Q; ++j) {
                double a = 0;
                for (int k = 0; k < Q; ++k)
                    if (tr->degree[k] <= max_degree) a += tr->Phi[k * Q + i] * tr->Phi[k * Q + j];
                F[i * Q + j] = float(a * tr->w[j]);
            }
        float* dF = nullptr;
        TCK(cudaMalloc(&dF, sizeof(float) * Q * Q));
        TCK(cudaMemcpyAsync(dF, F.data(), sizeof(float) * Q * Q, cudaMemcpyHostToDevice, tr->stream));
        k_filter_targets<<<unsigned((M + 127) / 128), 128, 0, tr->stream>>>(dR, M, Q, dF);
        TCK(cudaStreamSynchronize(tr->stream));
        cudaFree(dF);
    }
    k_data_stats<<<unsigned((M + 255) / 256), 256, 0, tr->stream>>>(dZ, dR, M, Q, tr->d_P, tr->d_w, acc);
    std::vector<double> a(Q + 1);
    TCK(cudaMemcpyAsync(a.data(), acc, sizeof(double) * (Q + 1), cudaMemcpyDeviceToHost, tr->stream));
    TCK(cudaStreamSynchronize(tr->stream));
    double amax = 0;
    for (int q = 0; q < Q; ++q) amax = std::max(amax, std::sqrt(a[q] / double(M)));
    for (int q = 0; q < Q; ++q) {
        const double rms = std::sqrt(a[q] / double(M));
        tr->s_in[q] = rms > 1e-6 * amax ? float(1.0 / rms) : 0.0f;   // conserved moments carry no signal
    }
    tr->sigma = float(std::sqrt(a[Q] / double(M)));
    if (!(tr->sigma > 0)) tr->sigma = 1.0f;
    TCK(cudaMemcpyAsync(tr->d_sin, tr->s_in.data(), sizeof(float) * Q, cudaMemcpyHostToDevice, tr->stream));
    k_normalise<<<unsigned((M * Q + 255) / 256), 256, 0, tr->stream>>>(dZ, dR, M, Q, tr->d_sin, 1.0f / tr->sigma,
                                                                       tr->d_X, tr->d_Y);
    TCK(cudaStreamSynchronize(tr->stream));
    cudaFree(dZ);
    cudaFree(dR);
    cudaFree(acc);
    tr->M = M;
    return SLLBM_OK;
}

int sllbm_train_scales(const sllbm_trainer* tr, float* s_in, float* sigma) {
    if (!tr) return SLLBM_ERR_ARG;
    if (s_in) std::memcpy(s_in, tr->s_in.data(), sizeof(float) * tr->Q);
    if (sigma) *sigma = tr->sigma;
    return SLLBM_OK;
}

int sllbm_train_grads(sllbm_trainer* tr, int64_t offset, int32_t count, float* grads, float* loss) {
    if (!tr || !tr->d_X || offset < 0 || count <= 0 || offset + count > tr->M) return SLLBM_ERR_ARG;
    cudaSetDevice(tr->device);
    const int n = n_params(tr->Q);
    TCK(cudaMemsetAsync(tr->d_grad, 0, sizeof(float) * n, tr->stream));
    TCK(cudaMemsetAsync(tr->d_loss, 0, sizeof(float), tr->stream));
    int rc = launch_batch(tr, offset, count, count);
    if (rc) return rc;
    if (grads) TCK(cudaMemcpyAsync(grads, tr->d_grad, sizeof(float) * n, cudaMemcpyDeviceToHost, tr->stream));
    float l = 0;
    int st = 0;
    TCK(cudaMemcpyAsync(&l, tr->d_loss, sizeof(float), cudaMemcpyDeviceToHost, tr->stream));
    TCK(cudaMemcpyAsync(&st, tr->d_status, sizeof(int), cudaMemcpyDeviceToHost, tr->stream));
    TCK(cudaMemsetAsync(tr->d_grad, 0, sizeof(float) * n, tr->stream));
    TCK(cudaStreamSynchronize(tr->stream));
    if (st) return tfail(tr, SLLBM_ERR_CUDA, "a tensor-core wait of the trainer ran out (status " + std::to_string(st) + ")");
    if (loss) *loss = l / float(count);
    return SLLBM_OK;
}

int sllbm_train_epoch(sllbm_trainer* tr, int32_t batch, float lr, float* loss) {
    if (!tr || !tr->d_X || batch <= 0 || !(lr > 0)) return SLLBM_ERR_ARG;
    cudaSetDevice(tr->device);
    const int n = n_params(tr->Q);
    int b1, W2, b2, W3, b3;
    offsets(tr->Q, b1, W2, b2, W3, b3);
    TCK(cudaMemsetAsync(tr->d_loss, 0, sizeof(float), tr->stream));
    for (int64_t off = 0; off + batch <= tr->M; off += batch) {
        int rc = launch_batch(tr, off, batch, batch);
        if (rc) return rc;
        ++tr->t;
        const float c1 = 1.0f - std::pow(0.9f, float(tr->t));
        const float c2 = 1.0f - std::pow(0.999f, float(tr->t));
        k_adam<<<(n + 255) / 256, 256, 0, tr->stream>>>(tr->d_p, tr->d_pr, tr->d_grad, tr->d_m, tr->d_v, n, 0, b1, W2,
                                                        b2, W3, b3, lr, c1, c2);
        TCK(cudaGetLastError());
    }
    float l = 0;
    int st = 0;
    TCK(cudaMemcpyAsync(&l, tr->d_loss, sizeof(float), cudaMemcpyDeviceToHost, tr->stream));
    TCK(cudaMemcpyAsync(&st, tr->d_status, sizeof(int), cudaMemcpyDeviceToHost, tr->stream));
    TCK(cudaStreamSynchronize(tr->stream));
    if (st) return tfail(tr, SLLBM_ERR_CUDA, "a tensor-core wait of the trainer ran out (status " + std::to_string(st) + ")");
    const int64_t nb = tr->M / batch;
    if (loss) *loss = nb > 0 ? l / float(nb * batch) : 0.f;
    return SLLBM_OK;
}

int sllbm_train_params(const sllbm_trainer* tr, float* params) {
    if (!tr || !params) return SLLBM_ERR_ARG;
    cudaSetDevice(tr->device);
    if (cudaMemcpy(params, tr->d_p, sizeof(float) * n_params(tr->Q), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SLLBM_ERR_CUDA;
    return SLLBM_OK;
}

int sllbm_train_set_params(sllbm_trainer* tr, const float* params) {
    if (!tr || !params) return SLLBM_ERR_ARG;
    cudaSetDevice(tr->device);
    const int n = n_params(tr->Q);
    int b1, W2, b2, W3, b3;
    offsets(tr->Q, b1, W2, b2, W3, b3);
    if (cudaMemcpy(tr->d_p, params, sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess) return SLLBM_ERR_CUDA;
    k_round_params<<<(n + 255) / 256, 256, 0, tr->stream>>>(tr->d_p, tr->d_pr, n, b1, W2, b2, W3, b3);
    return cudaStreamSynchronize(tr->stream) == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

// BF16 weights (W1 | W2 | W3 as bit patterns) and FP32 biases (b1 | b2 | b3)
int sllbm_train_export(const sllbm_trainer* tr, uint16_t* w_bf16, float* biases) {
    if (!tr) return SLLBM_ERR_ARG;
    cudaSetDevice(tr->device);
    const int Q = tr->Q, n = n_params(Q);
    std::vector<float> pr(n);
    if (cudaMemcpy(pr.data(), tr->d_pr, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SLLBM_ERR_CUDA;
    int b1, W2, b2, W3, b3;
    offsets(Q, b1, W2, b2, W3, b3);
    auto bits = [](float f) {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return uint16_t(u >> 16);   // already rounded to BF16
    };
    if (w_bf16) {
        int k = 0;
        for (int p = 0; p < b1; ++p) w_bf16[k++] = bits(pr[p]);
        for (int p = W2; p < b2; ++p) w_bf16[k++] = bits(pr[p]);
        for (int p = W3; p < b3; ++p) w_bf16[k++] = bits(pr[p]);
    }
    if (biases) {
        int k = 0;
        for (int p = b1; p < W2; ++p) biases[k++] = pr[p];
        for (int p = b2; p < W3; ++p) biases[k++] = pr[p];
        for (int p = b3; p < n; ++p) biases[k++] = pr[p];
    }
    return SLLBM_OK;
}

}  // extern "C"
