// Flow statistics as device reductions over node planes of constant y index
// (the homogeneous directions x and z of the channel and the mixing layer):
// Reynolds averages are arithmetic means over a plane (Sec. 4.3), so one
// block per plane sums, in FP64, the moments the Favre averages and the
// Reynolds stresses need.  The derived profiles are formed on the host.
#include "sllbm_internal.h"

namespace sllbm {

// per plane j: means of rho, rho u_a, u_a, T, rho T, rho u_a u_b (a <= b)
template <int D>
__global__ void __launch_bounds__(128) k_plane_sums(const double* __restrict__ rho, const double* __restrict__ u,
                                                    const double* __restrict__ T, int N0, int N1, int N2,
                                                    double* __restrict__ out, int accumulate) {
    constexpr int K = 3 + 2 * D + D * (D + 1) / 2;
    __shared__ double sh[K][128];
    const int j = blockIdx.x;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    const int64_t M = int64_t(N0) * N2;
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x) {
        const int64_t kx = m % N0, kz = m / N0;
        const int64_t n = kx + int64_t(N0) * (j + int64_t(N1) * kz);
        const double r = rho[n], t = T[n];
        double v[D];
#pragma unroll
        for (int d = 0; d < D; ++d) v[d] = u[n * D + d];
        int k = 0;
        acc[k++] += r;
#pragma unroll
        for (int d = 0; d < D; ++d) acc[k++] += r * v[d];
#pragma unroll
        for (int d = 0; d < D; ++d) acc[k++] += v[d];
        acc[k++] += t;
        acc[k++] += r * t;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) acc[k++] += r * v[a] * v[b];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = 64; s > 0; s >>= 1) {
        if (int(threadIdx.x) < s)
#pragma unroll
            for (int k = 0; k < K; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < K) {
        const double v = sh[threadIdx.x][0] / double(M);
        double& o = out[int64_t(j) * K + threadIdx.x];
        o = accumulate ? o + v : v;   // accumulate: running sums over time of the plane means
    }
}

// C_P = (rho T - p0) / denom at the nodes of plane j, x fastest then z
__global__ void k_plane_cp(const double* __restrict__ rho, const double* __restrict__ T, int N0, int N1, int N2,
                           int j, double p0, double denom, double* __restrict__ out) {
    const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (m >= int64_t(N0) * N2) return;
    const int64_t kx = m % N0, kz = m / N0;
    const int64_t n = kx + int64_t(N0) * (j + int64_t(N1) * kz);
    out[m] = (rho[n] * T[n] - p0) / denom;
}

int plane_stat_count(int D) { return 3 + 2 * D + D * (D + 1) / 2; }

int launch_plane_sums(const double* rho, const double* u, const double* T, int D, int N0, int N1, int N2,
                      double* out, int accumulate, cudaStream_t s) {
    if (N1 <= 0) return SLLBM_ERR_ARG;
    if (D == 2)
        k_plane_sums<2><<<N1, 128, 0, s>>>(rho, u, T, N0, N1, N2, out, accumulate);
    else if (D == 3)
        k_plane_sums<3><<<N1, 128, 0, s>>>(rho, u, T, N0, N1, N2, out, accumulate);
    else
        return SLLBM_ERR_ARG;
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

int launch_plane_cp(const double* rho, const double* T, int N0, int N1, int N2, int j, double p0, double denom,
                    double* out, cudaStream_t s) {
    const int64_t M = int64_t(N0) * N2;
    if (M <= 0) return SLLBM_ERR_ARG;
    k_plane_cp<<<unsigned((M + 255) / 256), 256, 0, s>>>(rho, T, N0, N1, N2, j, p0, denom, out);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

}  // namespace sllbm
