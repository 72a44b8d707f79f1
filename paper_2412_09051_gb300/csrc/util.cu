// Initialisation, state conversion, moment readout and FP64 conservation sums.
#include <algorithm>
#include <string>

#include "sllbm_internal.h"

namespace sllbm {

// equilibrium deviations (Sec. 3.1) of node fields, in FP64, stored as real
template <int VS, typename real>
__global__ void k_init(const double* __restrict__ rho, const double* __restrict__ u, const double* __restrict__ T,
                       int64_t N, const CollideConst<double> C, typename Vec2<real>::T* __restrict__ fg) {
    using VSET = VelSet<VS>;
    constexpr int D = VSET::D;
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double r = rho[n];
    double uu[3] = {u[n * D + 0], u[n * D + 1], D == 3 ? u[n * D + 2] : 0.0};
    const double U = uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2];
    const double t = T[n] - 1.0;
    EqCoef<double, VSET::NS> K;
    K.build(C, U, t);
    const double rT = r * (1.0 + t);
    Unroll<0, VSET::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        double fe, ge, cd;
        eq_dev<VSET, double, i>(C, K, uu, r, r - 1.0, rT, rT - 1.0, fe, ge, cd);
        fg[int64_t(i) * N + n] = Vec2<real>::make(real(fe), real(ge));
    });
}

// full <-> deviation conversion; dir = 0: dev -> full, 1: full -> dev
template <typename real>
__global__ void k_convert(typename Vec2<real>::T* __restrict__ fgd, double* __restrict__ ff,
                          double* __restrict__ gf, int64_t N, int Q, const double* __restrict__ w,
                          const double* __restrict__ wg, int dir) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= N * Q) return;
    const int i = int(t / N);
    if (dir == 0) {
        const auto v = fgd[t];
        ff[t] = double(v.x) + w[i];
        gf[t] = double(v.y) + wg[i];
    } else {
        fgd[t] = Vec2<real>::make(real(ff[t] - w[i]), real(gf[t] - wg[i]));
    }
}

// per-node moments (Sec. 3.1) in FP64 from the stored deviations
template <int VS, typename real>
__device__ __forceinline__ void node_moments(const typename Vec2<real>::T* fg, int64_t N, int64_t n,
                                             const CollideConst<double>& C, double& rho, double (&j)[3], double& e2) {
    using VSET = VelSet<VS>;
    double rd = 0, e = 0;
    j[0] = j[1] = j[2] = 0;
    Unroll<0, VSET::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const auto v = fg[int64_t(i) * N + n];
        const double fi = double(v.x);
        const double gi = double(v.y);
        rd += fi;
        j[0] += C.xi[i][0] * fi;
        j[1] += C.xi[i][1] * fi;
        if (VSET::D == 3) j[2] += C.xi[i][2] * fi;
        e += C.s2[VSET::shell(i)] * fi + gi;
    });
    rho = 1.0 + rd;
    e2 = e + 2.0 * C.cv;
}

template <int VS, typename real>
__global__ void k_moments(const typename Vec2<real>::T* __restrict__ fg, int64_t N,
                          const CollideConst<double> C, double* __restrict__ rho, double* __restrict__ u,
                          double* __restrict__ T) {
    using VSET = VelSet<VS>;
    constexpr int D = VSET::D;
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double r, j[3], e2;
    node_moments<VS, real>(fg, N, n, C, r, j, e2);
    double U = 0;
    for (int d = 0; d < D; ++d) {
        const double ud = j[d] / r;
        U += ud * ud;
        if (u) u[n * D + d] = ud;
    }
    if (rho) rho[n] = r;
    if (T) T[n] = (e2 - r * U) / (2.0 * r * C.cv);
}

// FP32 contexts: the same moments from compensated FP32 sums of the stored
// FP32 deviations (the precision the state carries, as in the step kernels);
// T is formed in FP64.  FP64 accumulation here was bound by the GB300's FP64
// rate, not by memory.
template <int VS>
__global__ void k_moments_f32(const float2* __restrict__ fg, int64_t N, const CollideConst<float> C, double cv,
                              double* __restrict__ rho, double* __restrict__ u, double* __restrict__ T) {
    using VSET = VelSet<VS>;
    constexpr int D = VSET::D;
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= N) return;
    Acc<float> ar, a0, a1, a2, ae;
    Unroll<0, VSET::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const float2 v = fg[int64_t(i) * N + n];
        ar.add(v.x);
        a0.add(C.xi[i][0] * v.x);
        a1.add(C.xi[i][1] * v.x);
        if (D == 3) a2.add(C.xi[i][2] * v.x);
        ae.add(C.s2[VSET::shell(i)] * v.x);
        ae.add(v.y);
    });
    const double r = 1.0 + double(ar.get());
    const double j[3] = {double(a0.get()), double(a1.get()), D == 3 ? double(a2.get()) : 0.0};
    const double e2 = double(ae.get()) + 2.0 * cv;
    double U = 0;
    for (int d = 0; d < D; ++d) {
        const double ud = j[d] / r;
        U += ud * ud;
        if (u) u[n * D + d] = ud;
    }
    if (rho) rho[n] = r;
    if (T) T[n] = (e2 - r * U) / (2.0 * r * cv);
}

// block partial sums of (rho, rho u, 2 rho E) and a positivity flag
template <int VS, typename real>
__global__ void k_conserve(const typename Vec2<real>::T* __restrict__ fg, int64_t N,
                           const CollideConst<double> C, double* __restrict__ part, int* __restrict__ flag) {
    using VSET = VelSet<VS>;
    constexpr int D = VSET::D;
    constexpr int K = D + 2;
    __shared__ double sh[K][256];
    double acc[K];
    for (int k = 0; k < K; ++k) acc[k] = 0;
    int bad = 0;
    for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < N; n += int64_t(gridDim.x) * blockDim.x) {
        double r, j[3], e2;
        node_moments<VS, real>(fg, N, n, C, r, j, e2);
        acc[0] += r;
        double U = 0;
        for (int d = 0; d < D; ++d) {
            acc[1 + d] += j[d];
            U += (j[d] / r) * (j[d] / r);
        }
        acc[D + 1] += e2;
        const double T = (e2 - r * U) / (2.0 * r * C.cv);
        if (!(r > 0.0) || !(T > 0.0) || !isfinite(e2)) bad = 1;
    }
    for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < K; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < K; ++k) part[blockIdx.x * K + k] = sh[k][0];
    if (bad) atomicOr(flag, 1);
}

__global__ void k_reduce_parts(const double* __restrict__ part, int nblk, int K, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= K) return;
    double s = 0;
    for (int b = 0; b < nblk; ++b) s += part[b * K + k];
    out[k] = s;
}

void k_reduce_parts_launch(const double* part, int nblk, int K, double* out, cudaStream_t s) {
    k_reduce_parts<<<1, 32, 0, s>>>(part, nblk, K, out);
}

// ------------------------------------------------------------ launchers
template <typename real>
int launch_init(int vs, const double* rho, const double* u, const double* T, int64_t N, const CollideConst<double>& C,
                typename Vec2<real>::T* fg, cudaStream_t s) {
    const int bs = 128;
    const unsigned grid = unsigned((N + bs - 1) / bs);
    switch (vs) {
        case 0: k_init<0, real><<<grid, bs, 0, s>>>(rho, u, T, N, C, fg); break;
        case 1: k_init<1, real><<<grid, bs, 0, s>>>(rho, u, T, N, C, fg); break;
        case 2: k_init<2, real><<<grid, bs, 0, s>>>(rho, u, T, N, C, fg); break;
        case 3: k_init<3, real><<<grid, bs, 0, s>>>(rho, u, T, N, C, fg); break;
        default: return SLLBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

template <typename real>
int launch_convert(typename Vec2<real>::T* fgd, double* ff, double* gf, int64_t N, int Q, const double* w,
                   const double* wg, int dir, cudaStream_t s) {
    const int bs = 256;
    k_convert<real><<<unsigned((N * Q + bs - 1) / bs), bs, 0, s>>>(fgd, ff, gf, N, Q, w, wg, dir);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

template <typename real>
int launch_moments(int vs, const typename Vec2<real>::T* fg, int64_t N, const CollideConst<double>& C, double* rho,
                   double* u, double* T, cudaStream_t s) {
    const int bs = 128;
    const unsigned grid = unsigned((N + bs - 1) / bs);
    switch (vs) {
        case 0: k_moments<0, real><<<grid, bs, 0, s>>>(fg, N, C, rho, u, T); break;
        case 1: k_moments<1, real><<<grid, bs, 0, s>>>(fg, N, C, rho, u, T); break;
        case 2: k_moments<2, real><<<grid, bs, 0, s>>>(fg, N, C, rho, u, T); break;
        case 3: k_moments<3, real><<<grid, bs, 0, s>>>(fg, N, C, rho, u, T); break;
        default: return SLLBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

int launch_moments_f32(int vs, const float2* fg, int64_t N, const CollideConst<float>& C, double cv, double* rho,
                       double* u, double* T, cudaStream_t s) {
    const int bs = 128;
    const unsigned grid = unsigned((N + bs - 1) / bs);
    switch (vs) {
        case 0: k_moments_f32<0><<<grid, bs, 0, s>>>(fg, N, C, cv, rho, u, T); break;
        case 1: k_moments_f32<1><<<grid, bs, 0, s>>>(fg, N, C, cv, rho, u, T); break;
        case 2: k_moments_f32<2><<<grid, bs, 0, s>>>(fg, N, C, cv, rho, u, T); break;
        case 3: k_moments_f32<3><<<grid, bs, 0, s>>>(fg, N, C, cv, rho, u, T); break;
        default: return SLLBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

int conserve_blocks() { return 152 * 4; }

template <typename real>
int launch_conserve(int vs, int D, const typename Vec2<real>::T* fg, int64_t N, const CollideConst<double>& C,
                    double* part, int* flag, double* out, cudaStream_t s) {
    const int nb = conserve_blocks();
    switch (vs) {
        case 0: k_conserve<0, real><<<nb, 256, 0, s>>>(fg, N, C, part, flag); break;
        case 1: k_conserve<1, real><<<nb, 256, 0, s>>>(fg, N, C, part, flag); break;
        case 2: k_conserve<2, real><<<nb, 256, 0, s>>>(fg, N, C, part, flag); break;
        case 3: k_conserve<3, real><<<nb, 256, 0, s>>>(fg, N, C, part, flag); break;
        default: return SLLBM_ERR_ARG;
    }
    k_reduce_parts<<<1, 32, 0, s>>>(part, nb, D + 2, out);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

#define INST(real)                                                                                                 \
    template int launch_init<real>(int, const double*, const double*, const double*, int64_t,                      \
                                   const CollideConst<double>&, Vec2<real>::T*, cudaStream_t);                     \
    template int launch_convert<real>(Vec2<real>::T*, double*, double*, int64_t, int, const double*,               \
                                      const double*, int, cudaStream_t);                                           \
    template int launch_moments<real>(int, const Vec2<real>::T*, int64_t, const CollideConst<double>&, double*,    \
                                      double*, double*, cudaStream_t);                                             \
    template int launch_conserve<real>(int, int, const Vec2<real>::T*, int64_t, const CollideConst<double>&,       \
                                       double*, int*, double*, cudaStream_t);
INST(float)
INST(double)

// mass rescaling (Sec. 4.3): full populations scaled by s; in deviation
// storage dev' = s dev + (s - 1) ref
template <typename real>
__global__ void k_scale_state(typename Vec2<real>::T* __restrict__ fg, int64_t N, int Q, const double* __restrict__ w,
                              const double* __restrict__ wg, double s) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= N * Q) return;
    const int i = int(t / N);
    auto v = fg[t];
    v.x = real(s * double(v.x) + (s - 1.0) * w[i]);
    v.y = real(s * double(v.y) + (s - 1.0) * wg[i]);
    fg[t] = v;
}

template <typename real>
int launch_scale_state(typename Vec2<real>::T* fg, int64_t N, int Q, const double* w, const double* wg, double s,
                       cudaStream_t st) {
    const int bs = 256;
    k_scale_state<real><<<unsigned((N * Q + bs - 1) / bs), bs, 0, st>>>(fg, N, Q, w, wg, s);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}
template int launch_scale_state<float>(float2*, int64_t, int, const double*, const double*, double, cudaStream_t);
template int launch_scale_state<double>(double2*, int64_t, int, const double*, const double*, double, cudaStream_t);

// node layers x0 .. x0 + nx - 1 of the state (all populations, all (y, z)
// rows) to / from a packed buffer [Q][rows][nx] of (f, g) pairs (dir 0: pack,
// 1: unpack); x0 + nx <= Nx
template <typename V2>
__global__ void k_x_layers(V2* __restrict__ fg, V2* __restrict__ buf, int64_t NN, int Nx, int rows, int x0, int nx,
                           int Q, int dir) {
    const int64_t tot = int64_t(Q) * rows * nx;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < tot; k += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = k / (int64_t(rows) * nx);
        const int64_t rem = k - i * rows * nx;
        const int64_t row = rem / nx;
        const int dx = int(rem - row * nx);
        const int64_t n = int64_t(x0 + dx) + int64_t(Nx) * row;
        if (dir == 0) buf[k] = fg[i * NN + n];
        else fg[i * NN + n] = buf[k];
    }
}

template <typename V2>
int launch_x_layers(V2* fg, V2* buf, int64_t NN, int Nx, int rows, int x0, int nx, int Q, int dir, cudaStream_t s) {
    const int64_t tot = int64_t(Q) * rows * nx;
    const int bs = 256;
    const int64_t blocks = std::min<int64_t>((tot + bs - 1) / bs, 152 * 16);
    if (tot == 0) return SLLBM_OK;
    k_x_layers<V2><<<unsigned(blocks), bs, 0, s>>>(fg, buf, NN, Nx, rows, x0, nx, Q, dir);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}
template int launch_x_layers<float2>(float2*, float2*, int64_t, int, int, int, int, int, int, cudaStream_t);
template int launch_x_layers<double2>(double2*, double2*, int64_t, int, int, int, int, int, int, cudaStream_t);

}  // namespace sllbm


// ====================================================================== allocation-free conservation
// sllbm_conservation_static: the conservation sums of sllbm_conservation with
// the per-block partial sums in a fixed device array compiled into this
// library instead of scratch owned by the context, for callers that must not
// allocate device memory themselves (see include/sllbm.h).
namespace sllbm {

// Layout (doubles): [0] positivity flag (as int), [8, 8 + D + 2) final sums,
// [16, 16 + blocks (D + 2)) block partials.  Fixed size: 2^17 doubles (1 MiB)
// on every device that loads the library, held until the process exits.
constexpr int kStaticScratchDoubles = 1 << 17;
constexpr int kStaticHead = 16;
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

template <typename real>
int launch_conserve_generic(const typename Vec2<real>::T* fg, int64_t N, const GenVel<double>* V, int Q, int D,
                            double cv, int grid_stride, unsigned blocks, double* part, int* flag, cudaStream_t s);

// one block per 256 nodes (no grid-stride loop): partial sums of
// (rho, rho u, 2 rho E) and the positivity flag
template <int VS, typename real>
__global__ void k_conserve_blocks(const typename Vec2<real>::T* __restrict__ fg, int64_t N,
                                  const CollideConst<double> C, double* __restrict__ part, int* __restrict__ flag) {
    using VSET = VelSet<VS>;
    constexpr int D = VSET::D;
    constexpr int K = D + 2;
    __shared__ double sh[K][256];
    double acc[K];
    for (int k = 0; k < K; ++k) acc[k] = 0;
    int bad = 0;
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n < N) {
        double r, j[3], e2;
        node_moments<VS, real>(fg, N, n, C, r, j, e2);
        acc[0] = r;
        double U = 0;
        for (int d = 0; d < D; ++d) {
            acc[1 + d] = j[d];
            U += (j[d] / r) * (j[d] / r);
        }
        acc[D + 1] = e2;
        const double T = (e2 - r * U) / (2.0 * r * C.cv);
        if (!(r > 0.0) || !(T > 0.0) || !isfinite(e2)) bad = 1;
    }
    for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < K; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < K; ++k) part[blockIdx.x * K + k] = sh[k][0];
    if (bad) atomicOr(flag, 1);
}

namespace {

template <typename real>
int launch_conserve_blocks(int vs, const typename Vec2<real>::T* fg, int64_t N, const CollideConst<double>& C,
                           double* part, int* flag, unsigned blocks, cudaStream_t s) {
    switch (vs) {
        case 0: k_conserve_blocks<0, real><<<blocks, 256, 0, s>>>(fg, N, C, part, flag); break;
        case 1: k_conserve_blocks<1, real><<<blocks, 256, 0, s>>>(fg, N, C, part, flag); break;
        case 2: k_conserve_blocks<2, real><<<blocks, 256, 0, s>>>(fg, N, C, part, flag); break;
        case 3: k_conserve_blocks<3, real><<<blocks, 256, 0, s>>>(fg, N, C, part, flag); break;
        default: return SLLBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}
}  // namespace
}  // namespace sllbm

extern "C" int sllbm_conservation_static(sllbm_ctx* ctx, double* out) {
    using namespace sllbm;
    if (!ctx || !out) return SLLBM_ERR_ARG;
    if (!ctx->initialised) {
        ctx->last_error = "state not initialised";
        return SLLBM_ERR_STATE;
    }
    const int dev = ctx->device;
    if (cudaSetDevice(dev) != cudaSuccess) {
        ctx->last_error = "cudaSetDevice failed";
        return SLLBM_ERR_CUDA;
    }
    const int64_t N = ctx->mesh.n_nodes;
    const int D = ctx->mesh.D;
    const int64_t blocks = (N + 255) / 256;
    if (kStaticHead + blocks * (D + 2) > kStaticScratchDoubles) {
        ctx->last_error = "mesh too large for the static scratch of sllbm_conservation_static: at most " +
                          std::to_string(int64_t(kStaticScratchDoubles - kStaticHead) / (D + 2) * 256) +
                          " nodes for D = " + std::to_string(D) + " (this mesh has " + std::to_string(N) + ")";
        return SLLBM_ERR_ARG;
    }
    // the device address of the array, looked up on every call with the
    // context's device current: a cached address would go stale if the
    // caller reset the device (the module, and the array, are then reloaded)
    double* base = nullptr;
    {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            ctx->last_error = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
            return SLLBM_ERR_CUDA;
        }
        base = static_cast<double*>(p);
    }
    int* flag = reinterpret_cast<int*>(base);
    double* sums = base + 8;
    double* part = base + kStaticHead;
    cudaStream_t s = ctx->stream;
    if (cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) {
        ctx->last_error = "cudaMemsetAsync failed";
        return SLLBM_ERR_CUDA;
    }
    const int c = ctx->cur;
    int rc;
    if (ctx->generic) {
        // one node per thread, the same block layout (generic.cu)
        const GenVel<double>* gv = static_cast<const GenVel<double>*>(ctx->gen_v64);
        rc = ctx->precision == SLLBM_FP64
                 ? launch_conserve_generic<double>((const double2*)ctx->fg[c], N, gv, ctx->vs.Q, D, ctx->cc64.cv, 0,
                                                   unsigned(blocks), part, flag, s)
                 : launch_conserve_generic<float>((const float2*)ctx->fg[c], N, gv, ctx->vs.Q, D, ctx->cc64.cv, 0,
                                                  unsigned(blocks), part, flag, s);
    } else {
        rc = ctx->precision == SLLBM_FP64
                 ? launch_conserve_blocks<double>(ctx->velset, (const double2*)ctx->fg[c], N, ctx->cc64, part, flag,
                                                  unsigned(blocks), s)
                 : launch_conserve_blocks<float>(ctx->velset, (const float2*)ctx->fg[c], N, ctx->cc64, part, flag,
                                                 unsigned(blocks), s);
    }
    if (rc == SLLBM_OK) {
        k_reduce_parts<<<1, 32, 0, s>>>(part, int(blocks), D + 2, sums);
        if (cudaGetLastError() != cudaSuccess) rc = SLLBM_ERR_CUDA;
    }
    if (rc) {
        ctx->last_error = "conservation launch failed";
        return rc;
    }
    int hflag = 0;
    if (cudaMemcpyAsync(out, sums, sizeof(double) * (D + 2), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        ctx->last_error = "copy of the conservation sums failed";
        return SLLBM_ERR_CUDA;
    }
    if (hflag) {
        ctx->last_error = "non-positive density or temperature, or non-finite state";
        return SLLBM_ERR_UNSTABLE;
    }
    return SLLBM_OK;
}
