// Generic velocity sets (D3Q125, caller-supplied sets; Sec. 3.2): the step,
// initialisation, moment and conservation kernels with the number of
// velocities known at run time and the per-velocity constants in a device
// table (GenVel).  The arithmetic is that of collide_node / k_init /
// node_moments for the compiled sets, with the shell constants of velocity i
// taken from its own table entry.
//
// Step (gather streaming, one thread per arrival node): every velocity's
// streamed pair is interpolated from its departure record exactly as in
// k_step_gather and written to the node's column of the output buffer, which
// then serves as the node's scratch: the compensated moments read it back,
// the isothermal correction and the relaxation rewrite it in place, the
// quasi-equilibrium heat flux is added in a last pass.
#include "sllbm_internal.h"
#include "step_kernels.cuh"

namespace sllbm {

namespace {

// P1 = P_i - 1 of velocity v at the state (u, U = |u|^2, t = T - 1), and xi.u
template <typename real>
__device__ __forceinline__ real gen_p1(const GenVel<real>& v, const real (&u)[3], real U, real t, real& cd) {
    const real c = v.xi[0] * u[0] + v.xi[1] * u[1] + v.xi[2] * u[2];
    cd = c;
    const real k2 = real(0.5) - real(0.25) * U + real(0.25) * t * v.sC;
    const real k1 = real(1.0) - real(0.5) * U + real(0.5) * t * v.sB;
    const real k0 = -real(0.5) * U + real(0.125) * U * U + real(0.5) * t * v.sA - real(0.25) * (t * U) * v.sB +
                    real(0.125) * (t * t) * v.sE;
    return eq_poly1(c, k0, k1, k2);
}

template <typename real>
__device__ __forceinline__ GenVel<real> gen_load(const GenVel<real>* V, int i) {
    GenVel<real> v;
    const real* s = reinterpret_cast<const real*>(V + i);
    real* d = reinterpret_cast<real*>(&v);
#pragma unroll
    for (int k = 0; k < int(sizeof(GenVel<real>) / sizeof(real)); ++k) d[k] = __ldg(s + k);
    return v;
}

}  // namespace

template <typename real, int P, int D>
__global__ void __launch_bounds__(128) k_step_generic(const typename Vec2<real>::T* __restrict__ fg,
                                                      typename Vec2<real>::T* __restrict__ fgo,
                                                      const int32_t* __restrict__ code,
                                                      const real* __restrict__ gxi, const real* __restrict__ twt,
                                                      const StepGeom G, const CollideConst<real> C,
                                                      const GenVel<real>* __restrict__ V, int Q) {
    using V2 = typename Vec2<real>::T;
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes) return;
    const int64_t NN = G.n_nodes;
    const int N0 = G.N[0], N1 = G.N[1];
    const int C0 = G.cells[0], C1 = G.cells[1];
    real xh[P + 1], inv_den[P + 1];
#pragma unroll
    for (int a = 0; a <= P; ++a) xh[a] = real(-cospi(double(a) / P));
#pragma unroll
    for (int a = 0; a <= P; ++a) {
        double den = 1.0;
        for (int m = 0; m <= P; ++m)
            if (m != a) den *= (-cospi(double(a) / P) + cospi(double(m) / P));
        inv_den[a] = real(1.0 / den);
    }
    // ---- streaming (Sec. 3.1, 3.3): into the node's column of fgo
#pragma unroll 1
    for (int i = 0; i < Q; ++i) {
        const GenVel<real> v = gen_load(V, i);
        const int cw = __ldg(code + int64_t(i) * NN + n);
        const int kind = (cw >> 24) & 15;
        const int bid = SLLBM_CHK((cw >> 28) & 15, 2, G.status, SLLBM_DEV_BAD_REC) & 1;
        real sf, sg;
        if (kind == REC_EQ) {
            sf = v.eqf[bid];
            sg = v.eqg[bid];
        } else {
            const int cell =
                SLLBM_CHK(cw & 0xFFFFFF, C0 * C1 * (D == 3 ? G.cells[2] : 1), G.status, SLLBM_DEV_BAD_REC);
            int cc[3];
            cc[0] = cell % C0;
            cc[1] = (cell / C0) % C1;
            cc[2] = cell / (C0 * C1);
            int64_t off[3][P + 1];
            real wt[3][P + 1];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const real x = __ldg(gxi + (int64_t(i) * D + d) * NN + n);
                lagrange_w<P, real>(x, xh, inv_den, wt[d]);
                const int64_t stride = d == 0 ? 1 : (d == 1 ? int64_t(N0) : int64_t(N0) * N1);
#pragma unroll
                for (int a = 0; a <= P; ++a) {
                    int kk = cc[d] * P + a;
                    if (G.periodic[d]) kk = wrapi(kk, G.N[d]);
                    off[d][a] = SLLBM_CHK(kk, G.N[d], G.status, SLLBM_DEV_BAD_NODE) * stride;
                }
            }
            const bool bb = kind == REC_BB || kind == REC_BB_ISO;
            const int src = SLLBM_CHK(bb ? v.opp : i, Q, G.status, SLLBM_DEV_BAD_POP);
            const V2* p = fg + int64_t(src) * NN;
            sf = 0;
            sg = 0;
            if (D == 2) {
#pragma unroll
                for (int b = 0; b <= P; ++b) {
                    real tf = 0, tg = 0;
#pragma unroll
                    for (int a = 0; a <= P; ++a) {
                        const V2 q = __ldg(p + off[0][a] + off[1][b]);
                        tf += wt[0][a] * q.x;
                        tg += wt[0][a] * q.y;
                    }
                    sf += wt[1][b] * tf;
                    sg += wt[1][b] * tg;
                }
            } else {
#pragma unroll
                for (int c3 = 0; c3 <= P; ++c3) {
                    real uf = 0, ug = 0;
#pragma unroll
                    for (int b = 0; b <= P; ++b) {
                        real tf = 0, tg = 0;
#pragma unroll
                        for (int a = 0; a <= P; ++a) {
                            const V2 q = __ldg(p + off[0][a] + off[1][b] + off[2][c3]);
                            tf += wt[0][a] * q.x;
                            tg += wt[0][a] * q.y;
                        }
                        uf += wt[1][b] * tf;
                        ug += wt[1][b] * tg;
                    }
                    sf += wt[2][c3] * uf;
                    sg += wt[2][c3] * ug;
                }
            }
            if (bb) sf += v.mw[bid];
        }
        fgo[int64_t(i) * NN + n] = Vec2<real>::make(sf, sg);
    }
    V2* col = fgo + n;
    // ---- moments (compensated in FP32), in velocity order as collide_node
    Acc<real> arho, aj0, aj1, aj2, ae;
#pragma unroll 1
    for (int i = 0; i < Q; ++i) {
        const GenVel<real> v = gen_load(V, i);
        const V2 q = col[int64_t(i) * NN];
        arho.add(q.x);
        aj0.add(v.xi[0] * q.x);
        aj1.add(v.xi[1] * q.x);
        if (D == 3) aj2.add(v.xi[2] * q.x);
        ae.add(v.s2 * q.x);
        ae.add(q.y);
    }
    const real rho_d = arho.get();
    const real rho = real(1) + rho_d;
    const real inv_rho = real(1) / rho;
    const real u[3] = {aj0.get() * inv_rho, aj1.get() * inv_rho, D == 3 ? aj2.get() * inv_rho : real(0)};
    const real U = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    real t = (ae.get() - rho * U - real(2) * C.cv * rho_d) * inv_rho / (real(2) * C.cv);
    // ---- isothermal wall correction (Eq. thermalBC): f += f^eq(T_w) - f^eq(T)
    const real Tw = twt[n];
    if (!(Tw != Tw)) {
        const real tw = Tw - real(1);
        const real rT0 = rho * (real(1) + t), rT1 = rho * (real(1) + tw);
#pragma unroll 1
        for (int i = 0; i < Q; ++i) {
            const GenVel<real> v = gen_load(V, i);
            real cd;
            const real a0 = gen_p1(v, u, U, t, cd), a1 = gen_p1(v, u, U, tw, cd);
            const real f0 = v.w * (rho * a0 + rho_d), g0 = v.wg * (rT0 * a0 + (rT0 - real(1)));
            const real f1 = v.w * (rho * a1 + rho_d), g1 = v.wg * (rT1 * a1 + (rT1 - real(1)));
            V2 q = col[int64_t(i) * NN];
            q.x += f1 - f0;
            q.y += g1 - g0;
            col[int64_t(i) * NN] = q;
        }
        t = tw;
    }
    const real T = real(1) + t;
    // ---- relaxation times (tau = mu / (p dt) + 1/2, tau_Pr = (tau - 1/2)/Pr + 1/2)
    real mu = C.mu_ref;
    if (C.var_mu) mu *= pow(T * C.inv_T_ref, C.mu_exp);
    const real tau = mu / (rho * T * C.dt) + real(0.5);
    const real om = real(1) / tau;
    const real om_pr = real(1) / ((tau - real(0.5)) * C.inv_Pr + real(0.5));
    const real rhoT = rho * T;
    const real rhoT_d = rho_d + rho * t;
    // Kupershtokh exact-difference forcing (Sec. 4.3), du = F dt / rho
    real vv[3] = {u[0], u[1], u[2]};
    if (C.forced) {
        vv[0] = u[0] + C.force_dt[0] * inv_rho;
        vv[1] = u[1] + C.force_dt[1] * inv_rho;
        vv[2] = D == 3 ? u[2] + C.force_dt[2] * inv_rho : real(0);
    }
    const real VV = vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2];
    real q0 = 0, q1 = 0, q2 = 0;
#pragma unroll 1
    for (int i = 0; i < Q; ++i) {
        const GenVel<real> v = gen_load(V, i);
        real cd;
        const real P1 = gen_p1(v, u, U, t, cd);
        const real fe = v.w * (rho * P1 + rho_d);
        const real ge = v.wg * (rhoT * P1 + rhoT_d);
        V2 q = col[int64_t(i) * NN];
        const real fn = q.x - fe, gn = q.y - ge;
        // central heat flux (times 2): sum (xi - u) (|xi - u|^2 f^neq + g^neq)
        const real h = (v.s2 - real(2) * cd + U) * fn + gn;
        q0 += (v.xi[0] - u[0]) * h;
        q1 += (v.xi[1] - u[1]) * h;
        if (D == 3) q2 += (v.xi[2] - u[2]) * h;
        q.x -= om * fn;
        q.y -= om * gn;
        if (C.forced) {
            real cw;
            const real Pv = gen_p1(v, vv, VV, t, cw);
            const real fa = v.w * (rho * Pv + rho_d);
            q.x += fa - fe;
        }
        col[int64_t(i) * NN] = q;
    }
    if (C.quasi) {
        // g*_i = w_i xi_i . (2 q^neq), weighted by (1/tau - 1/tau_Pr)
        const real a = om - om_pr;
        q0 *= a;
        q1 *= a;
        q2 *= a;
#pragma unroll 1
        for (int i = 0; i < Q; ++i) {
            const GenVel<real> v = gen_load(V, i);
            real d = v.xi[0] * q0 + v.xi[1] * q1;
            if (D == 3) d += v.xi[2] * q2;
            V2 q = col[int64_t(i) * NN];
            q.y += v.w * d;
            col[int64_t(i) * NN] = q;
        }
    }
}

// equilibrium deviations of node fields (FP64), as k_init
template <typename real>
__global__ void k_init_generic(const double* __restrict__ rho, const double* __restrict__ u,
                               const double* __restrict__ T, int64_t N, const GenVel<double>* __restrict__ V, int Q,
                               int D, typename Vec2<real>::T* __restrict__ fg) {
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double r = rho[n];
    const double uu[3] = {u[n * D + 0], u[n * D + 1], D == 3 ? u[n * D + 2] : 0.0};
    const double U = uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2];
    const double t = T[n] - 1.0;
    const double rT = r * (1.0 + t);
    for (int i = 0; i < Q; ++i) {
        const GenVel<double> v = gen_load(V, i);
        double cd;
        const double P1 = gen_p1(v, uu, U, t, cd);
        fg[int64_t(i) * N + n] = Vec2<real>::make(real(v.w * (r * P1 + (r - 1.0))), real(v.wg * (rT * P1 + (rT - 1.0))));
    }
}

// per-node moments in FP64 from the stored deviations, as node_moments
template <typename real>
__device__ __forceinline__ void gen_node_moments(const typename Vec2<real>::T* fg, int64_t N, int64_t n,
                                                 const GenVel<double>* V, int Q, double& rho, double (&j)[3],
                                                 double& e) {
    double rd = 0;
    e = 0;
    j[0] = j[1] = j[2] = 0;
    for (int i = 0; i < Q; ++i) {
        const GenVel<double> v = gen_load(V, i);
        const auto q = fg[int64_t(i) * N + n];
        const double fi = double(q.x), gi = double(q.y);
        rd += fi;
        j[0] += v.xi[0] * fi;
        j[1] += v.xi[1] * fi;
        j[2] += v.xi[2] * fi;
        e += v.s2 * fi + gi;
    }
    rho = 1.0 + rd;
}

template <typename real>
__global__ void k_moments_generic(const typename Vec2<real>::T* __restrict__ fg, int64_t N,
                                  const GenVel<double>* __restrict__ V, int Q, int D, double cv,
                                  double* __restrict__ rho, double* __restrict__ u, double* __restrict__ T) {
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double r, j[3], e;
    gen_node_moments<real>(fg, N, n, V, Q, r, j, e);
    const double e2 = e + 2.0 * cv;
    double U = 0;
    for (int d = 0; d < D; ++d) {
        const double ud = j[d] / r;
        U += ud * ud;
        if (u) u[n * D + d] = ud;
    }
    if (rho) rho[n] = r;
    if (T) T[n] = (e2 - r * U) / (2.0 * r * cv);
}

// block partial sums of (rho, rho u, 2 rho E) and the positivity flag; with
// grid_stride == 0 one node per thread (the allocation-free variant's layout)
template <typename real>
__global__ void k_conserve_generic(const typename Vec2<real>::T* __restrict__ fg, int64_t N,
                                   const GenVel<double>* __restrict__ V, int Q, int D, double cv, int grid_stride,
                                   double* __restrict__ part, int* __restrict__ flag) {
    const int K = D + 2;
    __shared__ double sh[5][256];
    double acc[5] = {0, 0, 0, 0, 0};
    int bad = 0;
    const int64_t step = grid_stride ? int64_t(gridDim.x) * blockDim.x : int64_t(N) + 1;
    for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < N; n += step) {
        double r, j[3], e;
        gen_node_moments<real>(fg, N, n, V, Q, r, j, e);
        const double e2 = e + 2.0 * cv;
        acc[0] += r;
        double U = 0;
        for (int d = 0; d < D; ++d) {
            acc[1 + d] += j[d];
            U += (j[d] / r) * (j[d] / r);
        }
        acc[D + 1] += e2;
        const double Tn = (e2 - r * U) / (2.0 * r * cv);
        if (!(r > 0.0) || !(Tn > 0.0) || !isfinite(e2)) bad = 1;
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

// ------------------------------------------------------------ launchers
template <typename real>
int launch_step_generic(int p, int D, const StepLaunch<real>& L, const GenVel<real>* V, int Q) {
    const int bs = 128;
    const unsigned grid = unsigned((L.G.n_nodes + bs - 1) / bs);
#define GCASE(P, DD)                                                                                          \
    if (p == P && D == DD) {                                                                                  \
        k_step_generic<real, P, DD><<<grid, bs, 0, L.stream>>>(L.fg, L.fgo, L.code, L.gxi, L.tw, L.G, *L.C, V, Q); \
        return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;                                  \
    }
    GCASE(2, 2)
    GCASE(3, 2)
    GCASE(4, 2)
    GCASE(2, 3)
    GCASE(3, 3)
    GCASE(4, 3)
#undef GCASE
    return SLLBM_ERR_UNSUPPORTED;
}

template <typename real>
int launch_init_generic(const double* rho, const double* u, const double* T, int64_t N, const GenVel<double>* V,
                        int Q, int D, typename Vec2<real>::T* fg, cudaStream_t s) {
    const int bs = 128;
    k_init_generic<real><<<unsigned((N + bs - 1) / bs), bs, 0, s>>>(rho, u, T, N, V, Q, D, fg);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

template <typename real>
int launch_moments_generic(const typename Vec2<real>::T* fg, int64_t N, const GenVel<double>* V, int Q, int D,
                           double cv, double* rho, double* u, double* T, cudaStream_t s) {
    const int bs = 128;
    k_moments_generic<real><<<unsigned((N + bs - 1) / bs), bs, 0, s>>>(fg, N, V, Q, D, cv, rho, u, T);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

template <typename real>
int launch_conserve_generic(const typename Vec2<real>::T* fg, int64_t N, const GenVel<double>* V, int Q, int D,
                            double cv, int grid_stride, unsigned blocks, double* part, int* flag, cudaStream_t s) {
    k_conserve_generic<real><<<blocks, 256, 0, s>>>(fg, N, V, Q, D, cv, grid_stride, part, flag);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

#define GINST(real)                                                                                             \
    template int launch_step_generic<real>(int, int, const StepLaunch<real>&, const GenVel<real>*, int);       \
    template int launch_init_generic<real>(const double*, const double*, const double*, int64_t,               \
                                           const GenVel<double>*, int, int, Vec2<real>::T*, cudaStream_t);     \
    template int launch_moments_generic<real>(const Vec2<real>::T*, int64_t, const GenVel<double>*, int, int,  \
                                              double, double*, double*, double*, cudaStream_t);                \
    template int launch_conserve_generic<real>(const Vec2<real>::T*, int64_t, const GenVel<double>*, int, int, \
                                               double, int, unsigned, double*, int*, cudaStream_t);
GINST(float)
GINST(double)
#undef GINST

}  // namespace sllbm
