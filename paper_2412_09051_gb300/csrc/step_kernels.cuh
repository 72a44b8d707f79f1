// Fused SLLBM pull step: stream by interpolation at the departure point
// (Sec. 3.1 Eq. intf / streamed-value formula), boundary records (Sec. 3.3),
// moments, isothermal correction (Eq. thermalBC) and collision (Eq. 1), one
// thread per arrival node, all 2Q streamed values held in registers.
#pragma once
#include "sllbm_internal.h"

namespace sllbm {

template <typename real>
struct StepLaunch {
    const real* f;
    const real* g;
    real* fo;
    real* go;
    const ClassRec<real>* cls;      // structured mode
    const int32_t* code;            // gather mode
    const real* gxi;                // gather mode
    const real* tw;                 // per class / per node wall temperature (NaN: none)
    StepGeom G;
    const CollideConst<real>* C;    // host copy, passed by value to the kernel
    cudaStream_t stream;
};

__device__ __forceinline__ int wrapi(int k, int N) { return k >= N ? k - N : k; }

// ------------------------------------------------------------ structured
template <int VS, int P, typename real>
__global__ void __launch_bounds__(128) k_step_structured(const real* __restrict__ f, const real* __restrict__ g,
                                                         real* __restrict__ fo, real* __restrict__ go,
                                                         const ClassRec<real>* __restrict__ tab,
                                                         const real* __restrict__ twt, const StepGeom G,
                                                         const CollideConst<real> C) {
    using VSET = VelSet<VS>;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes) return;
    const int N0 = G.N[0], N1 = G.N[1];
    int k[3];
    k[0] = int(n % N0);
    k[1] = int((n / N0) % N1);
    k[2] = D == 3 ? int(n / (int64_t(N0) * N1)) : 0;
    int cl[3], home[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        cl[d] = (d < D && G.periodic[d]) ? k[d] % P : (d < D ? k[d] : 0);
        home[d] = k[d] / P;
    }
    const int cls = cl[0] + G.ncls[0] * (cl[1] + G.ncls[1] * cl[2]);
    const int64_t NN = G.n_nodes;
    real fs[Q], gs[Q];
    Unroll<0, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const ClassRec<real>& r = tab[i * G.n_classes + cls];
        const int meta = __ldg(&r.meta);
        const int kind = meta & 15;
        const int bid = (meta >> 4) & 15;
        if (kind == REC_EQ) {
            fs[i] = C.eqf[bid][i];
            gs[i] = C.eqg[bid][i];
            return;
        }
        const int src = meta >> 8;
        int64_t off[3][P + 1];
        real wt[3][P + 1];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            int c = __ldg(&r.cell[d]);
            if (G.periodic[d]) {
                c += home[d];
                c %= G.cells[d];
                if (c < 0) c += G.cells[d];
            }
            const int64_t stride = d == 0 ? 1 : (d == 1 ? int64_t(N0) : int64_t(N0) * N1);
#pragma unroll
            for (int a = 0; a <= P; ++a) {
                int kk = c * P + a;
                if (G.periodic[d]) kk = wrapi(kk, G.N[d]);
                off[d][a] = kk * stride;
                wt[d][a] = __ldg(&r.wt[d][a]);
            }
        }
        const real* fp = f + int64_t(src) * NN;
        const real* gp = g + int64_t(src) * NN;
        real sf = 0, sg = 0;
        if (D == 2) {
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                real tf = 0, tg = 0;
#pragma unroll
                for (int a = 0; a <= P; ++a) {
                    const int64_t o = off[0][a] + off[1][b];
                    tf += wt[0][a] * __ldg(fp + o);
                    tg += wt[0][a] * __ldg(gp + o);
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
                        const int64_t o = off[0][a] + off[1][b] + off[2][c3];
                        tf += wt[0][a] * __ldg(fp + o);
                        tg += wt[0][a] * __ldg(gp + o);
                    }
                    uf += wt[1][b] * tf;
                    ug += wt[1][b] * tg;
                }
                sf += wt[2][c3] * uf;
                sg += wt[2][c3] * ug;
            }
        }
        if (kind == REC_BB || kind == REC_BB_ISO) sf += C.mw[bid][i];
        fs[i] = sf;
        gs[i] = sg;
    });
    collide_node<VSET, real>(C, fs, gs, twt[cls]);
    Unroll<0, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        fo[int64_t(i) * NN + n] = fs[i];
        go[int64_t(i) * NN + n] = gs[i];
    });
}

// ------------------------------------------------------------ gather
template <int VS, int P, typename real>
__global__ void __launch_bounds__(128) k_step_gather(const real* __restrict__ f, const real* __restrict__ g,
                                                     real* __restrict__ fo, real* __restrict__ go,
                                                     const int32_t* __restrict__ code,
                                                     const real* __restrict__ gxi, const real* __restrict__ twt,
                                                     const StepGeom G, const CollideConst<real> C,
                                                     const int* __restrict__ opp_unused) {
    using VSET = VelSet<VS>;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes) return;
    const int64_t NN = G.n_nodes;
    const int N0 = G.N[0], N1 = G.N[1];
    const int C0 = G.cells[0], C1 = G.cells[1];
    // GLC nodes and inverse Lagrange denominators for order P
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
    real fs[Q], gs[Q];
    Unroll<0, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const int cw = __ldg(code + int64_t(i) * NN + n);
        const int kind = (cw >> 24) & 15;
        const int bid = (cw >> 28) & 15;
        if (kind == REC_EQ) {
            fs[i] = C.eqf[bid][i];
            gs[i] = C.eqg[bid][i];
            return;
        }
        const int cell = cw & 0xFFFFFF;
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
                off[d][a] = kk * stride;
            }
        }
        const int src = (kind == REC_BB || kind == REC_BB_ISO) ? C.opp[i] : i;
        const real* fp = f + int64_t(src) * NN;
        const real* gp = g + int64_t(src) * NN;
        real sf = 0, sg = 0;
        if (D == 2) {
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                real tf = 0, tg = 0;
#pragma unroll
                for (int a = 0; a <= P; ++a) {
                    const int64_t o = off[0][a] + off[1][b];
                    tf += wt[0][a] * __ldg(fp + o);
                    tg += wt[0][a] * __ldg(gp + o);
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
                        const int64_t o = off[0][a] + off[1][b] + off[2][c3];
                        tf += wt[0][a] * __ldg(fp + o);
                        tg += wt[0][a] * __ldg(gp + o);
                    }
                    uf += wt[1][b] * tf;
                    ug += wt[1][b] * tg;
                }
                sf += wt[2][c3] * uf;
                sg += wt[2][c3] * ug;
            }
        }
        if (kind == REC_BB || kind == REC_BB_ISO) sf += C.mw[bid][i];
        fs[i] = sf;
        gs[i] = sg;
    });
    collide_node<VSET, real>(C, fs, gs, twt[n]);
    Unroll<0, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        fo[int64_t(i) * NN + n] = fs[i];
        go[int64_t(i) * NN + n] = gs[i];
    });
}

template <int VS, int P, typename real>
int launch_step_structured(const StepLaunch<real>& L) {
    const int bs = 128;
    const int64_t grid = (L.G.n_nodes + bs - 1) / bs;
    k_step_structured<VS, P, real><<<unsigned(grid), bs, 0, L.stream>>>(L.f, L.g, L.fo, L.go, L.cls, L.tw, L.G, *L.C);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

template <int VS, int P, typename real>
int launch_step_gather(const StepLaunch<real>& L) {
    const int bs = 128;
    const int64_t grid = (L.G.n_nodes + bs - 1) / bs;
    k_step_gather<VS, P, real><<<unsigned(grid), bs, 0, L.stream>>>(L.f, L.g, L.fo, L.go, L.code, L.gxi, L.tw, L.G,
                                                                     *L.C, nullptr);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

#define SLLBM_EXTERN_STEP(VS, P, real)                                                   \
    extern template int launch_step_structured<VS, P, real>(const StepLaunch<real>&);    \
    extern template int launch_step_gather<VS, P, real>(const StepLaunch<real>&);

#define SLLBM_INSTANTIATE_STEP(VS, P, real)                                              \
    template int launch_step_structured<VS, P, real>(const StepLaunch<real>&);           \
    template int launch_step_gather<VS, P, real>(const StepLaunch<real>&);

}  // namespace sllbm
