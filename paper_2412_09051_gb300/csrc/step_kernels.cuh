// Fused SLLBM pull step: stream by interpolation at the departure point
// (Sec. 3.1 Eq. intf / streamed-value formula), boundary records (Sec. 3.3),
// moments, isothermal correction (Eq. thermalBC) and collision (Eq. 1), one
// thread per arrival node, all 2Q streamed values held in registers.
#pragma once
#include "mlp.cuh"
#include "bulk.cuh"
#include "checked.cuh"
#include "mlp_tc.cuh"
#include "sllbm_internal.h"

namespace sllbm {

template <typename real>
struct StepLaunch {
    const typename Vec2<real>::T* fg;    // interleaved (f, g) per population, [Q][N]
    typename Vec2<real>::T* fgo;
    const ClassRec<real>* cls;      // structured mode
    const TileRec<real>* tile;      // warp-tiled mode
    const int32_t* code;            // gather mode
    const real* gxi;                // gather mode
    const real* tw;                 // per class / per node wall temperature (NaN: none)
    const float* mlp_img;           // learned-collision image (mlp.cuh) or nullptr
    float* feat;                    // feature export [N][Q] or nullptr
    StepGeom G;
    const CollideConst<real>* C;    // host copy, passed by value to the kernel
    cudaStream_t stream;
    const void* tilep = nullptr;        // warp-tiled records of order P (TileRecP), P > 2
    const uint16_t* mlp_tc = nullptr;   // BF16 weight tiles of the tensor-core MLP (mlp_tc.cuh)
    int* status = nullptr;              // device status word (tensor-core MLP)
    const RowRec* row = nullptr;        // one-block-per-row records (FP32)
};

__device__ __forceinline__ int wrapi(int k, int N) { return k >= N ? k - N : k; }

// sum-factorised tensor-product interpolation of one (f, g) population from
// the (P+1)^D source nodes at p + off[0][a] + off[1][b] (+ off[2][c]):
// x first, then y, then z; loads and multiply-adds interleaved (no staging)
template <int D, int P, typename real, typename V2>
__device__ __forceinline__ void interp_direct(const V2* __restrict__ p, const int64_t (&off)[3][P + 1],
                                              const real (&wt)[3][P + 1], real& of, real& og) {
    real sf = 0, sg = 0;
#pragma unroll
    for (int c3 = 0; c3 <= (D == 3 ? P : 0); ++c3) {
        real uf = 0, ug = 0;
#pragma unroll
        for (int b = 0; b <= P; ++b) {
            real tf = 0, tg = 0;
#pragma unroll
            for (int a = 0; a <= P; ++a) {
                const V2 v = __ldg(p + off[0][a] + off[1][b] + (D == 3 ? off[2][c3] : 0));
                tf += wt[0][a] * v.x;
                tg += wt[0][a] * v.y;
            }
            uf += wt[1][b] * tf;
            ug += wt[1][b] * tg;
        }
        if (D == 3) {
            sf += wt[2][c3] * uf;
            sg += wt[2][c3] * ug;
        } else {
            sf = uf;
            sg = ug;
        }
    }
    of = sf;
    og = sg;
}

// ------------------------------------------------------------ structured
template <int VS, int P, typename real>
__global__ void __launch_bounds__(128) k_step_structured(const typename Vec2<real>::T* __restrict__ fg,
                                                         typename Vec2<real>::T* __restrict__ fgo,
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
        const ClassRec<real>& r = tab[i * G.n_classes + SLLBM_CHK(cls, G.n_classes, G.status, SLLBM_DEV_BAD_REC)];
        const int meta = __ldg(&r.meta);
        const int kind = meta & 15;
        const int bid = (meta >> 4) & 15;
        if (kind == REC_EQ) {
            fs[i] = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            gs[i] = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            return;
        }
        const int src = SLLBM_CHK(meta >> 8, Q, G.status, SLLBM_DEV_BAD_POP);
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
                off[d][a] = SLLBM_CHK(kk, G.N[d], G.status, SLLBM_DEV_BAD_NODE) * stride;
                wt[d][a] = __ldg(&r.wt[d][a]);
            }
        }
        const typename Vec2<real>::T* p = fg + int64_t(src) * NN;
        real sf = 0, sg = 0;
        if (D == 2) {
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                real tf = 0, tg = 0;
#pragma unroll
                for (int a = 0; a <= P; ++a) {
                    const auto v = __ldg(p + off[0][a] + off[1][b]);
                    tf += wt[0][a] * v.x;
                    tg += wt[0][a] * v.y;
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
                        const auto v = __ldg(p + off[0][a] + off[1][b] + off[2][c3]);
                        tf += wt[0][a] * v.x;
                        tg += wt[0][a] * v.y;
                    }
                    uf += wt[1][b] * tf;
                    ug += wt[1][b] * tg;
                }
                sf += wt[2][c3] * uf;
                sg += wt[2][c3] * ug;
            }
        }
        if (kind == REC_BB || kind == REC_BB_ISO) sf += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
        fs[i] = sf;
        gs[i] = sg;
    });
    collide_node<VSET, real>(C, fs, gs, twt[cls]);
    Unroll<0, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        fgo[int64_t(i) * NN + n] = Vec2<real>::make(fs[i], gs[i]);
    });
}

// ------------------------------------------------------------ structured, state in shared memory
// The per-class records of k_step_structured with a runtime velocity loop and
// the node's 2Q streamed values in shared memory ([2][Q][128] per block), for
// orders whose (P+1)^D taps per population make a fully unrolled body too
// large (3D, p = 4: 125 taps).  No block barrier: threads are independent.
template <int VS, int P, typename real>
__global__ void __launch_bounds__(128, 4) k_step_structured_smem(const typename Vec2<real>::T* __restrict__ fg,
                                                              typename Vec2<real>::T* __restrict__ fgo,
                                                              const ClassRec<real>* __restrict__ tab,
                                                              const real* __restrict__ twt, const StepGeom G,
                                                              const CollideConst<real> C) {
    using VSET = VelSet<VS>;
    using V2 = typename Vec2<real>::T;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    real* S = reinterpret_cast<real*>(dyn_smem);
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
    constexpr int stride = 128;                  // the launch block size
    real* Sf = S + threadIdx.x;
    real* Sg = S + Q * stride + threadIdx.x;
#pragma unroll 1
    for (int i = 0; i < Q; ++i) {
        const ClassRec<real>& r = tab[i * G.n_classes + SLLBM_CHK(cls, G.n_classes, G.status, SLLBM_DEV_BAD_REC)];
        const int meta = __ldg(&r.meta);
        const int kind = meta & 15;
        const int bid = (meta >> 4) & 15;
        real of, og;
        if (kind == REC_EQ) {
            of = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            og = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
        } else {
            int64_t off[3][P + 1];
            real wt[3][P + 1];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int c = d < D ? __ldg(&r.cell[d]) : 0;
                if (d < D && G.periodic[d]) {
                    c += home[d];
                    c %= G.cells[d];
                    if (c < 0) c += G.cells[d];
                }
                const int64_t st = d == 0 ? 1 : (d == 1 ? int64_t(N0) : int64_t(N0) * N1);
#pragma unroll
                for (int a = 0; a <= P; ++a) {
                    int kk = c * P + a;
                    if (d < D && G.periodic[d]) kk = wrapi(kk, G.N[d]);
                    off[d][a] = d < D ? SLLBM_CHK(kk, G.N[d], G.status, SLLBM_DEV_BAD_NODE) * st : 0;
                    wt[d][a] = d < D ? __ldg(&r.wt[d][a]) : real(0);
                }
            }
            interp_direct<D, P, real, V2>(fg + int64_t(SLLBM_CHK(meta >> 8, Q, G.status, SLLBM_DEV_BAD_POP)) * NN, off, wt, of, og);
            if (kind == REC_BB || kind == REC_BB_ISO) of += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
        }
        Sf[i * stride] = of;
        Sg[i * stride] = og;
    }
    collide_smem<VSET, real, V2, 128>(C, Sf, Sg, twt[cls], fgo + n, int(NN));
}

// ------------------------------------------------------------ gather
template <int VS, int P, typename real>
__global__ void __launch_bounds__(128) k_step_gather(const typename Vec2<real>::T* __restrict__ fg,
                                                     typename Vec2<real>::T* __restrict__ fgo,
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
            fs[i] = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            gs[i] = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            return;
        }
        const int cell = SLLBM_CHK(cw & 0xFFFFFF, C0 * C1 * (D == 3 ? G.cells[2] : 1), G.status, SLLBM_DEV_BAD_REC);
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
        const int src = SLLBM_CHK((kind == REC_BB || kind == REC_BB_ISO) ? C.opp[i] : i, Q, G.status, SLLBM_DEV_BAD_POP);
        const typename Vec2<real>::T* p = fg + int64_t(src) * NN;
        real sf = 0, sg = 0;
        if (D == 2) {
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                real tf = 0, tg = 0;
#pragma unroll
                for (int a = 0; a <= P; ++a) {
                    const auto v = __ldg(p + off[0][a] + off[1][b]);
                    tf += wt[0][a] * v.x;
                    tg += wt[0][a] * v.y;
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
                        const auto v = __ldg(p + off[0][a] + off[1][b] + off[2][c3]);
                        tf += wt[0][a] * v.x;
                        tg += wt[0][a] * v.y;
                    }
                    uf += wt[1][b] * tf;
                    ug += wt[1][b] * tg;
                }
                sf += wt[2][c3] * uf;
                sg += wt[2][c3] * ug;
            }
        }
        if (kind == REC_BB || kind == REC_BB_ISO) sf += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
        fs[i] = sf;
        gs[i] = sg;
    });
    collide_node<VSET, real>(C, fs, gs, twt[n]);
    Unroll<0, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        fgo[int64_t(i) * NN + n] = Vec2<real>::make(fs[i], gs[i]);
    });
}

// ------------------------------------------------------------ warp-tiled (P = 2)
// One warp owns W = 32 - 2H consecutive x-nodes of one (y, z) row plus H halo
// nodes on each side.  For every velocity the y and z factors of the
// tensor-product Lagrange stencil are the same for the whole warp (x is
// periodic and uniform, the class differs only by the x parity), so each lane
// loads its own x-column of the (P+1)^(D-1) source rows (coalesced) and
// contracts them with the y/z weights; the x factor is then applied with warp
// shuffles from the neighbouring lanes (offsets within [-H, H], checked at
// setup).  Only lanes H .. H+W-1 store.
// MLPM: 0 plain collision, 1 learned correction on CUDA cores, 2 export of
// the MLP features (the tensor-core correction runs in k_step_tiled_smem_tc).
template <int VS, int H, typename real, int MLPM>
__global__ void __launch_bounds__(128) k_step_tiled(const typename Vec2<real>::T* __restrict__ fg,
                                                    typename Vec2<real>::T* __restrict__ fgo,
                                                    const TileRec<real>* __restrict__ tab,
                                                    const real* __restrict__ twt, const StepGeom G,
                                                    const CollideConst<real> C, const float* __restrict__ mlp_img,
                                                    float* __restrict__ feat) {
    using VSET = VelSet<VS>;
    using V2 = typename Vec2<real>::T;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    constexpr int W = 32 - 2 * H;
    constexpr int NR = D == 3 ? 9 : 3;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    float* mlp_s = reinterpret_cast<float*>(dyn_smem);
    if (MLPM) mlp_load<Q, D>(mlp_img, mlp_s);        // whole block, before any early exit
    const int lane = threadIdx.x & 31;
    const int gw = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    const int Nx = G.N[0], N1 = G.N[1];
    const int tiles = (Nx + W - 1) / W;
    const int rows = D == 3 ? N1 * G.N[2] : N1;
    if (gw >= tiles * rows) return;              // whole warps only
    const int row = gw / tiles;
    const int x0 = (gw - row * tiles) * W;
    const int ky = row % N1;
    const int kz = D == 3 ? row / N1 : 0;
    int kx = (x0 - H + lane) % Nx;
    if (kx < 0) kx += Nx;
    const bool store = lane >= H && lane < H + W && (x0 + lane - H) < Nx;
    const int NN = int(G.n_nodes);
    const int plane = Nx * N1;
    const int n = kx + Nx * ky + plane * kz;
    const bool py = G.periodic[1] != 0;
    const int cls = (kx & 1) + G.ncls[0] * ((py ? (ky & 1) : ky) + G.ncls[1] * (D == 3 ? (kz & 1) : 0));
    // rows near a periodic y / z seam need wrapped offsets (warp-uniform)
    const bool seam = (py && (ky < 3 || ky >= N1 - 3)) || (D == 3 && (kz < 3 || kz >= G.N[2] - 3));
    const V2* base = fg + n;
    real fs[Q], gs[Q];
    Unroll<0, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const TileRec<real>* r = tab + i * G.n_classes + SLLBM_CHK(cls, G.n_classes, G.status, SLLBM_DEV_BAD_REC);
        const int4 h0 = __ldg(reinterpret_cast<const int4*>(r));
        const int kind = h0.x & 15;
        const int bid = (h0.x >> 4) & 15;
        if (kind == REC_EQ) {
            fs[i] = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            gs[i] = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            return;
        }
        int rel[12];
        {
            const int4 a0 = __ldg(reinterpret_cast<const int4*>(r) + 1);
            const int4 a1 = __ldg(reinterpret_cast<const int4*>(r) + 2);
            const int4 a2 = __ldg(reinterpret_cast<const int4*>(r) + 3);
            rel[0] = a0.x; rel[1] = a0.y; rel[2] = a0.z; rel[3] = a0.w;
            rel[4] = a1.x; rel[5] = a1.y; rel[6] = a1.z; rel[7] = a1.w;
            rel[8] = a2.x;
        }
        if (seam) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const int dy = ((h0.z >> (4 * (k % 3))) & 15) - 8;
                const int dz = D == 3 ? ((h0.z >> (12 + 4 * (k / 3))) & 15) - 8 : 0;
                int ty = ky + dy, tz = kz + dz;
                if (py) { ty += ty < 0 ? N1 : 0; ty -= ty >= N1 ? N1 : 0; }
                if (D == 3) { tz += tz < 0 ? G.N[2] : 0; tz -= tz >= G.N[2] ? G.N[2] : 0; }
                rel[k] = (ty - ky) * Nx + (tz - kz) * plane;
            }
        }
        const V2* p = base + SLLBM_CHK(h0.x >> 8, Q, G.status, SLLBM_DEV_BAD_POP) * NN;
        real sf = 0, sg = 0;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const V2 v = __ldg(p + SLLBM_CHK_REL(n, rel[k], NN, G.status));
            const real wk = __ldg(&r->rw[k]);
            sf += wk * v.x;
            sg += wk * v.y;
        }
        real of = 0, og = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int dl = min(31, max(0, lane + ((h0.y >> (4 * a)) & 15) - 8));
            const real wx = __ldg(&r->wx[a]);
            of += wx * __shfl_sync(0xffffffffu, sf, dl);
            og += wx * __shfl_sync(0xffffffffu, sg, dl);
        }
        if (kind == REC_BB || kind == REC_BB_ISO) of += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
        fs[i] = of;
        gs[i] = og;
    });
    if (MLPM) {
        real fneq[Q];
        collide_node<VSET, real>(C, fs, gs, twt[cls], fneq);
        const MlpView<Q, D> M(mlp_s);
        float z[Q];
        mlp_moments<Q, D, real>(M, fneq, z);
        if (MLPM == 2) {
            if (store)
#pragma unroll
                for (int k = 0; k < Q; ++k) feat[int64_t(n) * Q + k] = z[k];
        } else {
            mlp_correct<Q, D, real>(M, C, z, fs);
        }
    } else {
        collide_node<VSET, real>(C, fs, gs, twt[cls]);
    }
    if (store) {
        Unroll<0, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            fgo[i * NN + n] = Vec2<real>::make(fs[i], gs[i]);
        });
    }
}

// ------------------------------------------------------------ warp-tiled, state in shared memory
// Same streaming as k_step_tiled, but with runtime velocity loops and the
// node's 2Q streamed values in shared memory ([2][Q][blockDim] per block): a
// compact kernel body and a small register footprint, so more warps per SM
// hide the load latency.  Warps are independent (no block barrier).
template <int VS, typename real>
__global__ void __launch_bounds__(128, 4) k_step_tiled_smem(const typename Vec2<real>::T* __restrict__ fg,
                                                         typename Vec2<real>::T* __restrict__ fgo,
                                                         const TileRec<real>* __restrict__ tab,
                                                         const real* __restrict__ twt, const StepGeom G,
                                                         const CollideConst<real> C) {
    using VSET = VelSet<VS>;
    using V2 = typename Vec2<real>::T;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    constexpr int H = 3, W = 32 - 2 * H;
    constexpr int NR = D == 3 ? 9 : 3;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    real* S = reinterpret_cast<real*>(dyn_smem);
    const int lane = threadIdx.x & 31;
    const int gw = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    const int Nx = G.N[0], N1 = G.N[1];
    const int tiles = (Nx + W - 1) / W;
    const int rows = D == 3 ? N1 * G.N[2] : N1;
    if (gw >= tiles * rows) return;              // whole warps only
    const int row = gw / tiles;
    const int x0 = (gw - row * tiles) * W;
    const int ky = row % N1;
    const int kz = D == 3 ? row / N1 : 0;
    int kx = (x0 - H + lane) % Nx;
    if (kx < 0) kx += Nx;
    const bool store = lane >= H && lane < H + W && (x0 + lane - H) < Nx;
    const int NN = int(G.n_nodes);
    const int plane = Nx * N1;
    const int n = kx + Nx * ky + plane * kz;
    const bool py = G.periodic[1] != 0;
    const int cls = (kx & 1) + G.ncls[0] * ((py ? (ky & 1) : ky) + G.ncls[1] * (D == 3 ? (kz & 1) : 0));
    const bool seam = (py && (ky < 3 || ky >= N1 - 3)) || (D == 3 && (kz < 3 || kz >= G.N[2] - 3));
    constexpr int stride = 128;                  // the launch block size
    real* Sf = S + threadIdx.x;
    real* Sg = S + Q * stride + threadIdx.x;
    const V2* base = fg + n;
    // velocities in groups of GV: all record loads of a group, then all source
    // loads (unconditional: equilibrium records read a valid dummy address), then
    // the arithmetic, so GV velocities' memory latencies overlap
    constexpr int GV = 3;
#pragma unroll 1
    for (int i0 = 0; i0 < Q; i0 += GV) {
        TileRec<real> r[GV];
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const int i = min(i0 + u, Q - 1);
            const int4* src = reinterpret_cast<const int4*>(tab + i * G.n_classes + SLLBM_CHK(cls, G.n_classes, G.status, SLLBM_DEV_BAD_REC));
            int4* dst = reinterpret_cast<int4*>(&r[u]);
#pragma unroll
            for (int k = 0; k < int(sizeof(TileRec<real>) / 16); ++k) dst[k] = __ldg(src + k);
        }
        V2 v[GV][NR];
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            // equilibrium records carry zero offsets and their own velocity as
            // source, so their (unused) loads read a valid row
            const bool eq = (r[u].meta & 15) == REC_EQ;
            int rel[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) rel[k] = r[u].rel[k];
            if (seam && !eq) {
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const int dy = ((r[u].dyzp >> (4 * (k % 3))) & 15) - 8;
                    const int dz = D == 3 ? ((r[u].dyzp >> (12 + 4 * (k / 3))) & 15) - 8 : 0;
                    int ty = ky + dy, tz = kz + dz;
                    if (py) { ty += ty < 0 ? N1 : 0; ty -= ty >= N1 ? N1 : 0; }
                    if (D == 3) { tz += tz < 0 ? G.N[2] : 0; tz -= tz >= G.N[2] ? G.N[2] : 0; }
                    rel[k] = (ty - ky) * Nx + (tz - kz) * plane;
                }
            }
            const V2* p = base + SLLBM_CHK(r[u].meta >> 8, Q, G.status, SLLBM_DEV_BAD_POP) * NN;
#pragma unroll
            for (int k = 0; k < NR; ++k) v[u][k] = __ldg(p + SLLBM_CHK_REL(n, rel[k], NN, G.status));
        }
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const int i = i0 + u;
            if (i >= Q) break;
            const int kind = r[u].meta & 15;
            const int bid = (r[u].meta >> 4) & 15;
            real of, og;
            if (kind == REC_EQ) {
                of = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                og = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            } else {
                real sf = 0, sg = 0;
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    sf += r[u].rw[k] * v[u][k].x;
                    sg += r[u].rw[k] * v[u][k].y;
                }
                of = 0;
                og = 0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    // source lane; halo lanes may point outside the warp (the
                    // shuffle wraps) but their results are never stored
                    const int dl = lane + ((r[u].dxp >> (4 * a)) & 15) - 8;
                    of += r[u].wx[a] * __shfl_sync(0xffffffffu, sf, dl);
                    og += r[u].wx[a] * __shfl_sync(0xffffffffu, sg, dl);
                }
                if (kind == REC_BB || kind == REC_BB_ISO) of += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            }
            Sf[i * stride] = of;
            Sg[i * stride] = og;
        }
    }
    collide_smem<VSET, real, V2, 128>(C, Sf, Sg, twt[cls], store ? fgo + n : nullptr, NN);
}

template <int VS, typename real>
int launch_step_tiled_smem(const StepLaunch<real>& L) {
    constexpr int H = 3, W = 32 - 2 * H;
    constexpr int Q = VelSet<VS>::Q, D = VelSet<VS>::D;
    const int tiles = (L.G.N[0] + W - 1) / W;
    const int64_t rows = D == 3 ? int64_t(L.G.N[1]) * L.G.N[2] : L.G.N[1];
    const int64_t threads = int64_t(tiles) * rows * 32;
    const int bs = 128;
    const size_t smem = sizeof(real) * 2 * Q * bs;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_step_tiled_smem<VS, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    k_step_tiled_smem<VS, real><<<unsigned((threads + bs - 1) / bs), bs, smem, L.stream>>>(L.fg, L.fgo, L.tile, L.tw,
                                                                                         L.G, *L.C);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

template <int VS, typename real, int MLPM = 0>
int launch_step_tiled(const StepLaunch<real>& L) {
    constexpr int H = 3, W = 32 - 2 * H;
    constexpr int Q = VelSet<VS>::Q, D = VelSet<VS>::D;
    const int tiles = (L.G.N[0] + W - 1) / W;
    const int64_t rows = D == 3 ? int64_t(L.G.N[1]) * L.G.N[2] : L.G.N[1];
    const int64_t threads = int64_t(tiles) * rows * 32;
    const int bs = 128;   // = TC_M: the tensor-core MLP takes one node per TMEM lane
    const size_t smem = MLPM ? sizeof(float) * mlp_image_floats(Q, D) : 0;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_step_tiled<VS, H, real, MLPM>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    k_step_tiled<VS, H, real, MLPM><<<unsigned((threads + bs - 1) / bs), bs, smem, L.stream>>>(
        L.fg, L.fgo, L.tile, L.tw, L.G, *L.C, L.mlp_img, L.feat);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

// ------------------------------------------------------------ one block per periodic row
// The streaming and collision of k_step_tiled_smem with one block of NXB = Nx
// threads per (y, z) row of a periodic x axis: every lane is an output node
// (the warp tiles spend 6 of 32 lanes on halos), and the x factor reads the
// neighbouring nodes' row sums from a shared row buffer, double-buffered per
// group of velocities with one block barrier per group.
template <int VS, typename real, int NXB>
__global__ void __launch_bounds__(256, 2) k_step_row_smem(const typename Vec2<real>::T* __restrict__ fg,
                                                       typename Vec2<real>::T* __restrict__ fgo,
                                                       const RowRec* __restrict__ tab,
                                                       const real* __restrict__ twt, const StepGeom G,
                                                       const CollideConst<real> C) {
    using VSET = VelSet<VS>;
    using V2 = typename Vec2<real>::T;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    constexpr int NR = D == 3 ? 9 : 3;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    real* S = reinterpret_cast<real*>(dyn_smem);
    real* XB = S + 2 * Q * NXB;
    const int Nx = NXB, N1 = G.N[1];
    const int row = blockIdx.x;
    const int ky = row % N1;
    const int kz = D == 3 ? row / N1 : 0;
    const int kx = threadIdx.x;
    const int NN = int(G.n_nodes);
    const int plane = Nx * N1;
    const int n = kx + Nx * ky + plane * kz;
    const bool py = G.periodic[1] != 0;
    const int cls = (kx & 1) + G.ncls[0] * ((py ? (ky & 1) : ky) + G.ncls[1] * (D == 3 ? (kz & 1) : 0));
    const bool seam = (py && (ky < 3 || ky >= N1 - 3)) || (D == 3 && (kz < 3 || kz >= G.N[2] - 3));
    constexpr int stride = NXB;
    real* Sf = S + threadIdx.x;
    real* Sg = S + Q * stride + threadIdx.x;
    const V2* base = fg + n;
    constexpr int GV = 3;
    int grp = 0;
#pragma unroll 1
    for (int i0 = 0; i0 < Q; i0 += GV, ++grp) {
        RowRec r[GV];
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const int i = min(i0 + u, Q - 1);
            const int4* src = reinterpret_cast<const int4*>(tab + i * G.n_classes + SLLBM_CHK(cls, G.n_classes, G.status, SLLBM_DEV_BAD_REC));
            int4* dst = reinterpret_cast<int4*>(&r[u]);
#pragma unroll
            for (int k = 0; k < int(sizeof(RowRec) / 16); ++k) dst[k] = __ldg(src + k);
        }
        V2 v[GV][NR];
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const bool eq = (r[u].meta & 15) == REC_EQ;
            int rel[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) rel[k] = r[u].rel[k];
            if (seam && !eq) {
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const int dy = ((r[u].dyzp >> (4 * (k % 3))) & 15) - 8;
                    const int dz = D == 3 ? ((r[u].dyzp >> (12 + 4 * (k / 3))) & 15) - 8 : 0;
                    int ty = ky + dy, tz = kz + dz;
                    if (py) { ty += ty < 0 ? N1 : 0; ty -= ty >= N1 ? N1 : 0; }
                    if (D == 3) { tz += tz < 0 ? G.N[2] : 0; tz -= tz >= G.N[2] ? G.N[2] : 0; }
                    rel[k] = (ty - ky) * Nx + (tz - kz) * plane;
                }
            }
            const V2* p = base + SLLBM_CHK(r[u].meta >> 8, Q, G.status, SLLBM_DEV_BAD_POP) * NN;
#pragma unroll
            for (int k = 0; k < NR; ++k) v[u][k] = __ldg(p + SLLBM_CHK_REL(n, rel[k], NN, G.status));
        }
        real* xb = XB + (grp & 1) * (GV * 2 * NXB);
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            real sf = 0, sg = 0;
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                sf += r[u].rw[k] * v[u][k].x;
                sg += r[u].rw[k] * v[u][k].y;
            }
            xb[(2 * u) * NXB + threadIdx.x] = sf;
            xb[(2 * u + 1) * NXB + threadIdx.x] = sg;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const int i = i0 + u;
            if (i >= Q) break;
            const int kind = r[u].meta & 15;
            const int bid = (r[u].meta >> 4) & 15;
            real of = 0, og = 0;
            if (kind == REC_EQ) {
                of = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                og = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    int j = int(threadIdx.x) + ((r[u].dxp >> (4 * a)) & 15) - 8;
                    j += j < 0 ? NXB : (j >= NXB ? -NXB : 0);
                    j = SLLBM_CHK(j, NXB, G.status, SLLBM_DEV_BAD_SMEM);
                    of += r[u].wx[a] * xb[(2 * u) * NXB + j];
                    og += r[u].wx[a] * xb[(2 * u + 1) * NXB + j];
                }
                if (kind == REC_BB || kind == REC_BB_ISO) of += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            }
            Sf[i * stride] = of;
            Sg[i * stride] = og;
        }
    }
    collide_smem<VSET, real, V2, NXB>(C, Sf, Sg, twt[cls], fgo + n, NN);
}

template <int VS, typename real, int NXB>
int launch_step_row_smem(const StepLaunch<real>& L) {
    constexpr int Q = VelSet<VS>::Q, D = VelSet<VS>::D;
    const int rows = D == 3 ? L.G.N[1] * L.G.N[2] : L.G.N[1];
    const size_t smem = sizeof(real) * (2 * Q * NXB + 2 * 3 * 2 * NXB);
    cudaFuncSetAttribute(k_step_row_smem<VS, real, NXB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    static_assert(std::is_same<real, float>::value, "row records are FP32");
    if (!L.row) return SLLBM_ERR_ARG;
    k_step_row_smem<VS, real, NXB><<<rows, NXB, smem, L.stream>>>(L.fg, L.fgo, L.row, L.tw, L.G, *L.C);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

// ------------------------------------------------------------ one block per periodic row, source rows copied by the bulk-copy engine
// k_step_row_smem with the source rows staged in shared memory by the TMA
// bulk-copy engine instead of loaded by every thread.  On a periodic x axis
// the (p+1)^(D-1) source rows of a velocity, (ky + dy_b, kz + dz_c), are
// whole x rows of NXB nodes of one population (contiguous, NXB float2), and
// the y/z stencil is the same for both x parities (checked at setup), so the
// first warp issues NR row copies per velocity (one per lane and round) into
// one of NST stages, NST velocities ahead, completing on the stage's
// mbarrier; every thread then
// contracts its own column from shared memory (no per-thread addressing or
// gathers).  A stage is refilled after the block barrier that follows its
// use (velocities in groups of GV, one barrier per group as in
// k_step_row_smem).  Every wait is bounded: on a timeout the block records
// SLLBM_DEV_COPY_TIMEOUT, stops issuing and computing, waits (bounded) for
// the copies it issued and returns without storing.
template <int VS, typename real, int NXB, int NST>
__global__ void __launch_bounds__(NXB, (VelSet<VS>::D == 3 ? 256 : 512) / NXB)
    k_step_row_copy(const typename Vec2<real>::T* __restrict__ fg, typename Vec2<real>::T* __restrict__ fgo,
                    const TileRec<real>* __restrict__ tab, const real* __restrict__ twt, const StepGeom G,
                    const CollideConst<real> C, int* __restrict__ status) {
    using VSET = VelSet<VS>;
    using V2 = typename Vec2<real>::T;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    constexpr int NR = D == 3 ? 9 : 3;
    constexpr int GV = 3;
    static_assert(NST % GV == 0 && NST >= GV, "stages hold whole velocity groups");
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    V2* RB = reinterpret_cast<V2*>(dyn_smem);                          // [NST][NR][NXB] staged rows
    real* S = reinterpret_cast<real*>(RB + NST * NR * NXB);            // [f, g][Q][NXB] streamed state
    real* XB = S + 2 * Q * NXB;                                        // [2][GV][f, g][NXB] row sums
    uint64_t* bars = reinterpret_cast<uint64_t*>(XB + 2 * GV * 2 * NXB);   // [NST] + 1 that nothing completes
    const int N1 = G.N[1], N2 = D == 3 ? G.N[2] : 1;
    const int row = blockIdx.x;
    const int ky = row % N1;
    const int kz = D == 3 ? row / N1 : 0;
    const int NN = int(G.n_nodes);
    const int plane = NXB * N1;
    const int n = int(threadIdx.x) + NXB * ky + plane * kz;
    const bool py = G.periodic[1] != 0;
    const int cls0 = G.ncls[0] * ((py ? (ky & 1) : ky) + G.ncls[1] * (D == 3 ? (kz & 1) : 0));   // x parity 0
    const int cls = int(threadIdx.x & 1) + cls0;
    const uint32_t bar0 = smem_u32(bars);
    const uint32_t rb0 = smem_u32(RB);
    // producer (warp 0, all lanes): the copies of velocities [ib, ie), at most
    // NST of them; lane u < ie - ib arms the barrier of velocity ib + u, then
    // every lane issues one row copy per round
    auto issue = [&](int ib, int ie) {
        const int lane = int(threadIdx.x & 31);
        int meta = REC_EQ, dyzp = 0;
        if (lane < ie - ib) {
            const int i = ib + lane;
            const TileRec<real>* r = tab + i * G.n_classes + SLLBM_CHK(cls0, G.n_classes, G.status, SLLBM_DEV_BAD_REC);
            meta = __ldg(&r->meta);
            dyzp = __ldg(&r->dyzp);
            const uint32_t bar = bar0 + 8u * uint32_t(i % NST);
            if ((meta & 15) == REC_EQ) mbar_arrive(bar);            // equilibrium record: no source rows
            else mbar_arrive_expect_tx(bar, uint32_t(NR * NXB * sizeof(V2)));
        }
        __syncwarp();
#pragma unroll
        for (int round = 0; round < (NST * NR + 31) / 32; ++round) {
            const int c = round * 32 + lane;
            const int u = min(c / NR, 31), k = c - (c / NR) * NR;
            const int m = __shfl_sync(0xffffffffu, meta, u);
            const int d = __shfl_sync(0xffffffffu, dyzp, u);
            if (c < (ie - ib) * NR && (m & 15) != REC_EQ) {
                const int i = ib + u;
                int ty = ky + ((d >> (4 * (k % 3))) & 15) - 8;
                int tz = D == 3 ? kz + ((d >> (12 + 4 * (k / 3))) & 15) - 8 : 0;
                if (py) { ty += ty < 0 ? N1 : 0; ty -= ty >= N1 ? N1 : 0; }
                if (D == 3) { tz += tz < 0 ? N2 : 0; tz -= tz >= N2 ? N2 : 0; }
                ty = SLLBM_CHK(ty, N1, G.status, SLLBM_DEV_BAD_NODE);
                tz = SLLBM_CHK(tz, N2, G.status, SLLBM_DEV_BAD_NODE);
                const V2* src = fg + int64_t(SLLBM_CHK(m >> 8, Q, G.status, SLLBM_DEV_BAD_POP)) * NN +
                                (int64_t(tz) * N1 + ty) * NXB;
                bulk_g2s(rb0 + uint32_t(((i % NST) * NR + k) * NXB * sizeof(V2)), src, uint32_t(NXB * sizeof(V2)),
                         bar0 + 8u * uint32_t(i % NST));
            }
        }
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s <= NST; ++s) mbar_init(bar0 + 8u * uint32_t(s), 1);
    }
    __syncthreads();
    const long long lim = wait_limit(status);
    int issued = min(NST, Q);                   // velocities whose copies were issued (warp 0)
    if (threadIdx.x < 32) issue(0, issued);
    real* Sf = S + threadIdx.x;
    real* Sg = S + Q * NXB + threadIdx.x;
    int grp = 0, waited = 0;
    bool aborted = false;
#pragma unroll 1
    for (int i0 = 0; i0 < Q; i0 += GV, ++grp) {
        TileRec<real> r[GV];                    // meta / dxp / dyzp and the weights (no node offsets)
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const int i = min(i0 + u, Q - 1);
            const int4* src = reinterpret_cast<const int4*>(tab + i * G.n_classes +
                                                            SLLBM_CHK(cls, G.n_classes, G.status, SLLBM_DEV_BAD_REC));
            int4* dst = reinterpret_cast<int4*>(&r[u]);
            dst[0] = __ldg(src);
#pragma unroll
            for (int k = 4; k < 7; ++k) dst[k] = __ldg(src + k);
        }
        bool ok = true;
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const int i = i0 + u;
            if (i < Q) ok = mbar_wait(bar0 + 8u * uint32_t(i % NST), uint32_t((i / NST) & 1), lim) && ok;
        }
        // under a test limit (sllbm_debug_wait_limit) also wait on the barrier
        // that nothing completes, so that the wait runs out whatever the timing
        if (lim < kWaitLimit) ok = mbar_wait(bar0 + 8u * uint32_t(NST), 0, lim) && ok;
        if (ok) waited = min(i0 + GV, Q);
        real* xb = XB + (grp & 1) * (GV * 2 * NXB);
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const V2* rb = RB + ((i0 + u) % NST) * NR * NXB + threadIdx.x;
            real sf = 0, sg = 0;
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const V2 v = rb[k * NXB];
                sf += r[u].rw[k] * v.x;
                sg += r[u].rw[k] * v.y;
            }
            xb[(2 * u) * NXB + threadIdx.x] = sf;
            xb[(2 * u + 1) * NXB + threadIdx.x] = sg;
        }
        // block barrier and vote in one: every thread sees the same answer,
        // so the break is block-uniform (a shared flag written before the
        // barrier could be overwritten by a thread that is already a group
        // ahead before a slower thread has read it)
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        // the group's stages are free: refill them NST velocities ahead
        if (threadIdx.x < 32 && issued < Q) {
            const int ie = min(i0 + GV + NST, Q);
            issue(issued, ie);
            issued = ie;
        }
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const int i = i0 + u;
            if (i >= Q) break;
            const int kind = r[u].meta & 15;
            const int bid = (r[u].meta >> 4) & 15;
            real of = 0, og = 0;
            if (kind == REC_EQ) {
                of = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                og = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    int j = int(threadIdx.x) + ((r[u].dxp >> (4 * a)) & 15) - 8;
                    j += j < 0 ? NXB : (j >= NXB ? -NXB : 0);
                    j = SLLBM_CHK(j, NXB, G.status, SLLBM_DEV_BAD_SMEM);
                    of += r[u].wx[a] * xb[(2 * u) * NXB + j];
                    og += r[u].wx[a] * xb[(2 * u + 1) * NXB + j];
                }
                if (kind == REC_BB || kind == REC_BB_ISO) of += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            }
            Sf[i * NXB] = of;
            Sg[i * NXB] = og;
        }
    }
    if (aborted) {
        if (threadIdx.x == 0) {
            atomicOr(status, SLLBM_DEV_COPY_TIMEOUT);
            // wait (bounded, default limit) for the copies issued but not yet
            // waited for, so that none lands after the block has exited
            for (int i = waited; i < issued; ++i) mbar_wait(bar0 + 8u * uint32_t(i % NST), uint32_t((i / NST) & 1));
        }
        return;
    }
    collide_smem<VSET, real, V2, NXB>(C, Sf, Sg, twt[cls], fgo + n, NN);
}

template <int VS, typename real, int NXB, int NST>
int launch_step_row_copy(const StepLaunch<real>& L) {
    constexpr int Q = VelSet<VS>::Q, D = VelSet<VS>::D;
    constexpr int NR = D == 3 ? 9 : 3;
    if (!L.status) return SLLBM_ERR_ARG;
    const int rows = D == 3 ? L.G.N[1] * L.G.N[2] : L.G.N[1];
    const size_t smem = sizeof(typename Vec2<real>::T) * NST * NR * NXB + sizeof(real) * (2 * Q * NXB + 2 * 3 * 2 * NXB) +
                        sizeof(uint64_t) * (NST + 1);
    cudaFuncSetAttribute(k_step_row_copy<VS, real, NXB, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    k_step_row_copy<VS, real, NXB, NST><<<rows, NXB, smem, L.stream>>>(L.fg, L.fgo, L.tile, L.tw, L.G, *L.C, L.status);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

// ------------------------------------------------------------ one block per periodic row, order P
// k_step_tiled_p's order-P streaming with one block of NXB = Nx threads per
// (y, z) row (no halo lanes: the warp tiles spend 2P of 32 lanes on halos);
// the x factor reads the neighbouring nodes' row sums from a shared row
// buffer, double-buffered per pair of velocities with one block barrier per
// pair.
template <int VS, int P, typename real, int NXB>
__global__ void __launch_bounds__(256, 2) k_step_row_p(const typename Vec2<real>::T* __restrict__ fg,
                                                    typename Vec2<real>::T* __restrict__ fgo,
                                                    const TileRecP<real, P>* __restrict__ tab,
                                                    const real* __restrict__ twt, const StepGeom G,
                                                    const CollideConst<real> C) {
    using VSET = VelSet<VS>;
    using V2 = typename Vec2<real>::T;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    constexpr int NZ = D == 3 ? P + 1 : 1;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    real* S = reinterpret_cast<real*>(dyn_smem);
    real* XB = S + 2 * Q * NXB;                  // [2 buffers][2 velocities][f, g][NXB]
    const int Nx = NXB, N1 = G.N[1], N2 = D == 3 ? G.N[2] : 1;
    const int row = blockIdx.x;
    const int ky = row % N1;
    const int kz = row / N1;
    const int kx = threadIdx.x;
    const int NN = int(G.n_nodes);
    const int plane = Nx * N1;
    const int n = kx + Nx * ky + plane * kz;
    const bool py = G.periodic[1] != 0;
    const int cls = (kx % P) + G.ncls[0] * ((py ? (ky % P) : ky) + G.ncls[1] * (D == 3 ? (kz % P) : 0));
    constexpr int stride = NXB;
    real* Sf = S + threadIdx.x;
    real* Sg = S + Q * stride + threadIdx.x;
    const V2* base = fg + n;
    // velocities in pairs: both pairs' row sums go through one buffer of the
    // double-buffered row buffer with one block barrier per pair (equilibrium
    // records write zeros), so two uses of one buffer always have the other
    // buffer's barrier between them
#pragma unroll 1
    for (int i0 = 0, pr = 0; i0 < Q; i0 += 2, ++pr) {
        TileRecP<real, P> r[2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
            r[u] = tab[min(i0 + u, Q - 1) * G.n_classes + SLLBM_CHK(cls, G.n_classes, G.status, SLLBM_DEV_BAD_REC)];
        real* xb = XB + (pr & 1) * (2 * 2 * NXB);   // [u][f, g][NXB]
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            real sf = 0, sg = 0;
            if ((r[u].meta & 15) != REC_EQ && i0 + u < Q) {   // kind uniform over the row (checked at setup)
                int oy[P + 1], oz[NZ];
#pragma unroll
                for (int b = 0; b <= P; ++b) {
                    int ty = ky + ((r[u].dyp >> (4 * b)) & 15) - 8;
                    if (py) ty += ty < 0 ? N1 : (ty >= N1 ? -N1 : 0);
                    oy[b] = (ty - ky) * Nx;
                }
#pragma unroll
                for (int c = 0; c < NZ; ++c) {
                    int tz = kz + ((r[u].dzp >> (4 * c)) & 15) - 8;
                    tz += tz < 0 ? N2 : (tz >= N2 ? -N2 : 0);
                    oz[c] = D == 3 ? (tz - kz) * plane : 0;
                }
                const V2* p = base + SLLBM_CHK(r[u].meta >> 8, Q, G.status, SLLBM_DEV_BAD_POP) * NN;
#pragma unroll
                for (int c = 0; c < NZ; ++c) {
                    real tf = 0, tg = 0;
#pragma unroll
                    for (int b = 0; b <= P; ++b) {
                        const V2 v = __ldg(p + SLLBM_CHK_REL(n, oy[b] + oz[c], NN, G.status));
                        tf += r[u].wy[b] * v.x;
                        tg += r[u].wy[b] * v.y;
                    }
                    const real wz = D == 3 ? r[u].wz[c] : real(1);
                    sf += wz * tf;
                    sg += wz * tg;
                }
            }
            xb[(2 * u) * NXB + threadIdx.x] = sf;
            xb[(2 * u + 1) * NXB + threadIdx.x] = sg;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = i0 + u;
            if (i >= Q) break;
            const int kind = r[u].meta & 15;
            const int bid = (r[u].meta >> 4) & 15;
            real of = 0, og = 0;
            if (kind == REC_EQ) {
                of = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                og = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            } else {
#pragma unroll
                for (int a = 0; a <= P; ++a) {
                    int j = int(threadIdx.x) + ((r[u].dxp >> (4 * a)) & 15) - 8;
                    j += j < 0 ? NXB : (j >= NXB ? -NXB : 0);
                    j = SLLBM_CHK(j, NXB, G.status, SLLBM_DEV_BAD_SMEM);
                    of += r[u].wx[a] * xb[(2 * u) * NXB + j];
                    og += r[u].wx[a] * xb[(2 * u + 1) * NXB + j];
                }
                if (kind == REC_BB || kind == REC_BB_ISO) of += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            }
            Sf[i * stride] = of;
            Sg[i * stride] = og;
        }
    }
    collide_smem<VSET, real, V2, NXB>(C, Sf, Sg, twt[cls], fgo + n, NN);
}

template <int VS, int P, typename real, int NXB>
int launch_step_row_p(const StepLaunch<real>& L) {
    constexpr int Q = VelSet<VS>::Q, D = VelSet<VS>::D;
    if (!L.tilep) return SLLBM_ERR_ARG;
    const int rows = D == 3 ? L.G.N[1] * L.G.N[2] : L.G.N[1];
    const size_t smem = sizeof(real) * (2 * Q * NXB + 2 * 2 * 2 * NXB);
    cudaFuncSetAttribute(k_step_row_p<VS, P, real, NXB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    k_step_row_p<VS, P, real, NXB><<<rows, NXB, smem, L.stream>>>(
        L.fg, L.fgo, static_cast<const TileRecP<real, P>*>(L.tilep), L.tw, L.G, *L.C);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

// ------------------------------------------------------------ warp-tiled smem state + learned correction on tcgen05
// k_step_tiled_smem's streaming and shared-memory collision, then the learned
// correction on the tensor cores (mlp_tc.cuh).  The node state (f, g and
// f^neq, 3 Q x 128 values) lives in the shared-memory region of the MMA
// activation operands, which the network needs only after the collision, so a
// block takes 51 KB of shared memory and fits 4 per SM next to 4 x 128 TMEM
// columns.  Every thread of the block takes part (idle warps carry zeros).
template <int VS, typename real>
__global__ void __launch_bounds__(128, 4) k_step_tiled_smem_tc(const typename Vec2<real>::T* __restrict__ fg,
                                                            typename Vec2<real>::T* __restrict__ fgo,
                                                            const TileRec<real>* __restrict__ tab,
                                                            const real* __restrict__ twt, const StepGeom G,
                                                            const CollideConst<real> C,
                                                            const float* __restrict__ mlp_img,
                                                            const uint16_t* __restrict__ mlp_tc,
                                                            int* __restrict__ status) {
    using VSET = VelSet<VS>;
    using V2 = typename Vec2<real>::T;
    using L = MlpTc<VSET::Q, VSET::D>;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    constexpr int H = 3, W = 32 - 2 * H;
    constexpr int NR = D == 3 ? 9 : 3;
    constexpr int stride = 128;                  // the launch block size
    static_assert(3 * Q * stride * sizeof(real) <= 2 * L::A_BYTES, "node state fits the operand buffers");
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const uint32_t tbase = mlp_tc_setup<Q, D>(mlp_img, mlp_tc, dyn_smem);   // whole block
    real* S = reinterpret_cast<real*>(dyn_smem + L::OFF_AHI);
    const int lane = threadIdx.x & 31;
    const int gw = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    const int Nx = G.N[0], N1 = G.N[1];
    const int tiles = (Nx + W - 1) / W;
    const int rows = D == 3 ? N1 * G.N[2] : N1;
    const bool live = gw < tiles * rows;         // whole warps
    const int row = live ? gw / tiles : 0;
    const int x0 = (gw - row * tiles) * W;
    const int ky = row % N1;
    const int kz = D == 3 ? row / N1 : 0;
    int kx = (x0 - H + lane) % Nx;
    if (kx < 0) kx += Nx;
    const bool store = live && lane >= H && lane < H + W && (x0 + lane - H) < Nx;
    const int NN = int(G.n_nodes);
    const int plane = Nx * N1;
    const int n = kx + Nx * ky + plane * kz;
    const bool py = G.periodic[1] != 0;
    const int cls = (kx & 1) + G.ncls[0] * ((py ? (ky & 1) : ky) + G.ncls[1] * (D == 3 ? (kz & 1) : 0));
    const bool seam = (py && (ky < 3 || ky >= N1 - 3)) || (D == 3 && (kz < 3 || kz >= G.N[2] - 3));
    real* Sf = S + threadIdx.x;
    real* Sg = S + Q * stride + threadIdx.x;
    real* Sn = S + 2 * Q * stride + threadIdx.x;
    if (live) {
        const V2* base = fg + n;
        // velocities in groups of GV: all record loads of a group, then all source
        // loads (unconditional: equilibrium records read a valid dummy address), then
        // the arithmetic, so GV velocities' memory latencies overlap
        constexpr int GV = 3;
    #pragma unroll 1
        for (int i0 = 0; i0 < Q; i0 += GV) {
            TileRec<real> r[GV];
    #pragma unroll
            for (int u = 0; u < GV; ++u) {
                const int i = min(i0 + u, Q - 1);
                const int4* src = reinterpret_cast<const int4*>(tab + i * G.n_classes + SLLBM_CHK(cls, G.n_classes, G.status, SLLBM_DEV_BAD_REC));
                int4* dst = reinterpret_cast<int4*>(&r[u]);
    #pragma unroll
                for (int k = 0; k < int(sizeof(TileRec<real>) / 16); ++k) dst[k] = __ldg(src + k);
            }
            V2 v[GV][NR];
    #pragma unroll
            for (int u = 0; u < GV; ++u) {
                // equilibrium records carry zero offsets and their own velocity as
                // source, so their (unused) loads read a valid row
                const bool eq = (r[u].meta & 15) == REC_EQ;
                int rel[NR];
    #pragma unroll
                for (int k = 0; k < NR; ++k) rel[k] = r[u].rel[k];
                if (seam && !eq) {
    #pragma unroll
                    for (int k = 0; k < NR; ++k) {
                        const int dy = ((r[u].dyzp >> (4 * (k % 3))) & 15) - 8;
                        const int dz = D == 3 ? ((r[u].dyzp >> (12 + 4 * (k / 3))) & 15) - 8 : 0;
                        int ty = ky + dy, tz = kz + dz;
                        if (py) { ty += ty < 0 ? N1 : 0; ty -= ty >= N1 ? N1 : 0; }
                        if (D == 3) { tz += tz < 0 ? G.N[2] : 0; tz -= tz >= G.N[2] ? G.N[2] : 0; }
                        rel[k] = (ty - ky) * Nx + (tz - kz) * plane;
                    }
                }
                const V2* p = base + SLLBM_CHK(r[u].meta >> 8, Q, G.status, SLLBM_DEV_BAD_POP) * NN;
    #pragma unroll
                for (int k = 0; k < NR; ++k) v[u][k] = __ldg(p + SLLBM_CHK_REL(n, rel[k], NN, G.status));
            }
    #pragma unroll
            for (int u = 0; u < GV; ++u) {
                const int i = i0 + u;
                if (i >= Q) break;
                const int kind = r[u].meta & 15;
                const int bid = (r[u].meta >> 4) & 15;
                real of, og;
                if (kind == REC_EQ) {
                    of = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                    og = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                } else {
                    real sf = 0, sg = 0;
    #pragma unroll
                    for (int k = 0; k < NR; ++k) {
                        sf += r[u].rw[k] * v[u][k].x;
                        sg += r[u].rw[k] * v[u][k].y;
                    }
                    of = 0;
                    og = 0;
    #pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        // source lane; halo lanes may point outside the warp (the
                        // shuffle wraps) but their results are never stored
                        const int dl = lane + ((r[u].dxp >> (4 * a)) & 15) - 8;
                        of += r[u].wx[a] * __shfl_sync(0xffffffffu, sf, dl);
                        og += r[u].wx[a] * __shfl_sync(0xffffffffu, sg, dl);
                    }
                    if (kind == REC_BB || kind == REC_BB_ISO) of += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                }
                Sf[i * stride] = of;
                Sg[i * stride] = og;
            }
        }
        collide_smem<VSET, real, V2, 128, true>(C, Sf, Sg, twt[cls], static_cast<V2*>(nullptr), NN, Sn);
    }
    const MlpView<Q, D> M(reinterpret_cast<const float*>(dyn_smem + L::OFF_TAIL), typename MlpView<Q, D>::TailOnly{});
    float z[Q];
    real f[Q], g[Q];
    if (live) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f[i] = Sf[i * stride];
            g[i] = Sg[i * stride];
        }
        // z_k = sum_i Phi_ki f^neq_i, summed in i order as mlp_moments does,
        // with a runtime velocity loop (a small body for the instruction cache)
#pragma unroll
        for (int k = 0; k < Q; ++k) z[k] = 0.f;
#pragma unroll 1
        for (int i = 0; i < Q; ++i) {
            const float fn = float(Sn[i * stride]);
#pragma unroll
            for (int k = 0; k < Q; ++k) z[k] += M.phi[k * Q + i] * fn;
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f[i] = g[i] = real(0);
            z[i] = 0.f;
        }
    }
    __syncthreads();                             // node state read: the operand buffers are free
    mlp_correct_tc<Q, D, real>(M, C, dyn_smem, tbase, z, f, status);   // whole block; frees TMEM
    if (store) {
#pragma unroll
        for (int i = 0; i < Q; ++i) fgo[int64_t(i) * NN + n] = Vec2<real>::make(f[i], g[i]);
    }
}

template <int VS, typename real>
int launch_step_tiled_smem_tc(const StepLaunch<real>& L) {
    constexpr int H = 3, W = 32 - 2 * H;
    constexpr int Q = VelSet<VS>::Q, D = VelSet<VS>::D;
    if (!L.mlp_tc || !L.status || !L.mlp_img) return SLLBM_ERR_ARG;
    const int tiles = (L.G.N[0] + W - 1) / W;
    const int64_t rows = D == 3 ? int64_t(L.G.N[1]) * L.G.N[2] : L.G.N[1];
    const int64_t threads = int64_t(tiles) * rows * 32;
    const int bs = 128;   // = TC_M: one node per TMEM lane
    const size_t smem = size_t(MlpTc<Q, D>::SMEM);
    cudaFuncSetAttribute(k_step_tiled_smem_tc<VS, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    k_step_tiled_smem_tc<VS, real><<<unsigned((threads + bs - 1) / bs), bs, smem, L.stream>>>(
        L.fg, L.fgo, L.tile, L.tw, L.G, *L.C, L.mlp_img, L.mlp_tc, L.status);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

// ------------------------------------------------------------ warp-tiled, order P, state in shared memory
// The warp-tiled streaming of k_step_tiled_smem for order P cells: a warp owns
// W = 32 - 2P consecutive x-nodes of one (y, z) row plus P halo lanes per side;
// per velocity each lane loads its x-column of the (P+1)^(D-1) source rows,
// contracts them with the factorised y then z weights and takes the x factor
// from the P+1 neighbouring lanes by shuffles.  Source-row offsets are formed
// from the packed dy / dz with the periodic wrap (no seam special case).
// Requires every x class of a (y, z) class to share the record's kind, y/z
// cell and y/z weights (checked at setup), so branches are warp-uniform.
template <int VS, int P, typename real>
__global__ void __launch_bounds__(128, 4) k_step_tiled_p(const typename Vec2<real>::T* __restrict__ fg,
                                                      typename Vec2<real>::T* __restrict__ fgo,
                                                      const TileRecP<real, P>* __restrict__ tab,
                                                      const real* __restrict__ twt, const StepGeom G,
                                                      const CollideConst<real> C) {
    using VSET = VelSet<VS>;
    using V2 = typename Vec2<real>::T;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    constexpr int H = P, W = 32 - 2 * H;
    constexpr int NZ = D == 3 ? P + 1 : 1;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    real* S = reinterpret_cast<real*>(dyn_smem);
    const int lane = threadIdx.x & 31;
    const int gw = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    const int Nx = G.N[0], N1 = G.N[1], N2 = D == 3 ? G.N[2] : 1;
    const int tiles = (Nx + W - 1) / W;
    const int rows = N1 * N2;
    if (gw >= tiles * rows) return;              // whole warps only
    const int row = gw / tiles;
    const int x0 = (gw - row * tiles) * W;
    const int ky = row % N1;
    const int kz = row / N1;
    int kx = (x0 - H + lane) % Nx;
    if (kx < 0) kx += Nx;
    const bool store = lane >= H && lane < H + W && (x0 + lane - H) < Nx;
    const int NN = int(G.n_nodes);
    const int plane = Nx * N1;
    const int n = kx + Nx * ky + plane * kz;
    const bool py = G.periodic[1] != 0;
    const int cls = (kx % P) + G.ncls[0] * ((py ? (ky % P) : ky) + G.ncls[1] * (D == 3 ? (kz % P) : 0));
    constexpr int stride = 128;                  // the launch block size
    real* Sf = S + threadIdx.x;
    real* Sg = S + Q * stride + threadIdx.x;
    const V2* base = fg + n;
#pragma unroll 1
    for (int i = 0; i < Q; ++i) {
        const TileRecP<real, P> r = tab[i * G.n_classes + SLLBM_CHK(cls, G.n_classes, G.status, SLLBM_DEV_BAD_REC)];
        const int kind = r.meta & 15;
        const int bid = (r.meta >> 4) & 15;
        real of = 0, og = 0;
        if (kind == REC_EQ) {
            of = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            og = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
        } else {
            int oy[P + 1], oz[NZ];
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                int ty = ky + ((r.dyp >> (4 * b)) & 15) - 8;
                if (py) ty += ty < 0 ? N1 : (ty >= N1 ? -N1 : 0);
                oy[b] = (ty - ky) * Nx;
            }
#pragma unroll
            for (int c = 0; c < NZ; ++c) {
                int tz = kz + ((r.dzp >> (4 * c)) & 15) - 8;
                tz += tz < 0 ? N2 : (tz >= N2 ? -N2 : 0);
                oz[c] = D == 3 ? (tz - kz) * plane : 0;
            }
            const V2* p = base + SLLBM_CHK(r.meta >> 8, Q, G.status, SLLBM_DEV_BAD_POP) * NN;
            real sf = 0, sg = 0;
#pragma unroll
            for (int c = 0; c < NZ; ++c) {
                real tf = 0, tg = 0;
#pragma unroll
                for (int b = 0; b <= P; ++b) {
                    const V2 v = __ldg(p + SLLBM_CHK_REL(n, oy[b] + oz[c], NN, G.status));
                    tf += r.wy[b] * v.x;
                    tg += r.wy[b] * v.y;
                }
                const real wz = D == 3 ? r.wz[c] : real(1);
                sf += wz * tf;
                sg += wz * tg;
            }
#pragma unroll
            for (int a = 0; a <= P; ++a) {
                // halo lanes may read across the warp edge (the shuffle wraps);
                // their results are never stored
                const int dl = lane + ((r.dxp >> (4 * a)) & 15) - 8;
                of += r.wx[a] * __shfl_sync(0xffffffffu, sf, dl);
                og += r.wx[a] * __shfl_sync(0xffffffffu, sg, dl);
            }
            if (kind == REC_BB || kind == REC_BB_ISO) of += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
        }
        Sf[i * stride] = of;
        Sg[i * stride] = og;
    }
    collide_smem<VSET, real, V2, 128>(C, Sf, Sg, twt[cls], store ? fgo + n : nullptr, NN);
}

template <int VS, int P, typename real>
int launch_step_tiled_p(const StepLaunch<real>& L) {
    constexpr int W = 32 - 2 * P;
    constexpr int Q = VelSet<VS>::Q, D = VelSet<VS>::D;
    if (!L.tilep) return SLLBM_ERR_ARG;
    const int tiles = (L.G.N[0] + W - 1) / W;
    const int64_t rows = D == 3 ? int64_t(L.G.N[1]) * L.G.N[2] : L.G.N[1];
    const int64_t threads = int64_t(tiles) * rows * 32;
    const int bs = 128;
    const size_t smem = sizeof(real) * 2 * Q * bs;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_step_tiled_p<VS, P, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    k_step_tiled_p<VS, P, real><<<unsigned((threads + bs - 1) / bs), bs, smem, L.stream>>>(
        L.fg, L.fgo, static_cast<const TileRecP<real, P>*>(L.tilep), L.tw, L.G, *L.C);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

// ------------------------------------------------------------ gather, state in shared memory
// One departure record per (velocity, node) as in k_step_gather, with the
// node state in shared memory, runtime velocity loops and the records and
// source loads of GV velocities issued together (GV = 2 for up to 16 taps).
template <int VS, int P, typename real>
__global__ void __launch_bounds__(128, 4) k_step_gather_smem(const typename Vec2<real>::T* __restrict__ fg,
                                                          typename Vec2<real>::T* __restrict__ fgo,
                                                          const int32_t* __restrict__ code,
                                                          const real* __restrict__ gxi, const real* __restrict__ twt,
                                                          const StepGeom G, const CollideConst<real> C) {
    using VSET = VelSet<VS>;
    using V2 = typename Vec2<real>::T;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    constexpr int T1 = P + 1;
    constexpr int NT = D == 3 ? T1 * T1 * T1 : T1 * T1;
    constexpr int GV = NT <= 16 ? 2 : 1;
    constexpr bool STAGE = NT <= 32;             // else interpolate while loading (3D, p >= 3)
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    real* S = reinterpret_cast<real*>(dyn_smem);
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= G.n_nodes) return;                   // no block barrier in this kernel
    const int64_t NN = G.n_nodes;
    const int N0 = G.N[0], N1 = G.N[1];
    const int C0 = G.cells[0], C1 = G.cells[1];
    real xh[T1], inv_den[T1];
#pragma unroll
    for (int a = 0; a <= P; ++a) xh[a] = real(-cospi(double(a) / P));
#pragma unroll
    for (int a = 0; a <= P; ++a) {
        double den = 1.0;
        for (int m = 0; m <= P; ++m)
            if (m != a) den *= (-cospi(double(a) / P) + cospi(double(m) / P));
        inv_den[a] = real(1.0 / den);
    }
    constexpr int stride = 128;                  // the launch block size
    real* Sf = S + threadIdx.x;
    real* Sg = S + Q * stride + threadIdx.x;
    if constexpr (!STAGE) {
#pragma unroll 1
        for (int i = 0; i < Q; ++i) {
            const int cw = __ldg(code + int64_t(i) * NN + n);
            const int kind = (cw >> 24) & 15;
            const int bid = (cw >> 28) & 15;
            real of, og;
            if (kind == REC_EQ) {
                of = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                og = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            } else {
                const int cell = SLLBM_CHK(cw & 0xFFFFFF, C0 * C1 * (D == 3 ? G.cells[2] : 1), G.status, SLLBM_DEV_BAD_REC);
                int cc[3];
                cc[0] = cell % C0;
                cc[1] = (cell / C0) % C1;
                cc[2] = cell / (C0 * C1);
                int64_t off[3][T1];
                real wt[3][T1];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (d < D) {
                        lagrange_w<P, real>(__ldg(gxi + (int64_t(i) * D + d) * NN + n), xh, inv_den, wt[d]);
                    } else {
#pragma unroll
                        for (int a = 0; a <= P; ++a) wt[d][a] = real(0);
                    }
                    const int64_t st = d == 0 ? 1 : (d == 1 ? int64_t(N0) : int64_t(N0) * N1);
#pragma unroll
                    for (int a = 0; a <= P; ++a) {
                        int kk = cc[d] * P + a;
                        if (d < D && G.periodic[d]) kk = wrapi(kk, G.N[d]);
                        off[d][a] = d < D ? SLLBM_CHK(kk, G.N[d], G.status, SLLBM_DEV_BAD_NODE) * st : 0;
                    }
                }
                const int src = SLLBM_CHK((kind == REC_BB || kind == REC_BB_ISO) ? C.opp[i] : i, Q, G.status, SLLBM_DEV_BAD_POP);
                interp_direct<D, P, real, V2>(fg + int64_t(src) * NN, off, wt, of, og);
                if (kind == REC_BB || kind == REC_BB_ISO) of += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            }
            Sf[i * stride] = of;
            Sg[i * stride] = og;
        }
    } else
#pragma unroll 1
    for (int i0 = 0; i0 < Q; i0 += GV) {
        int cw[GV];
        real xr[GV][D];
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const int i = min(i0 + u, Q - 1);
            cw[u] = __ldg(code + int64_t(i) * NN + n);
#pragma unroll
            for (int d = 0; d < D; ++d) xr[u][d] = __ldg(gxi + (int64_t(i) * D + d) * NN + n);
        }
        V2 v[GV][NT];
        real wt[GV][D][T1];
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const int i = min(i0 + u, Q - 1);
            const int kind = (cw[u] >> 24) & 15;
            const bool eq = kind == REC_EQ;
            const int cell = SLLBM_CHK(eq ? 0 : (cw[u] & 0xFFFFFF), C0 * C1 * (D == 3 ? G.cells[2] : 1), G.status, SLLBM_DEV_BAD_REC);
            int cc[3];
            cc[0] = cell % C0;
            cc[1] = (cell / C0) % C1;
            cc[2] = cell / (C0 * C1);
            int64_t off[3][T1];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                lagrange_w<P, real>(xr[u][d], xh, inv_den, wt[u][d]);
                const int64_t st = d == 0 ? 1 : (d == 1 ? int64_t(N0) : int64_t(N0) * N1);
#pragma unroll
                for (int a = 0; a <= P; ++a) {
                    int kk = cc[d] * P + a;
                    if (G.periodic[d]) kk = wrapi(kk, G.N[d]);
                    off[d][a] = SLLBM_CHK(kk, G.N[d], G.status, SLLBM_DEV_BAD_NODE) * st;
                }
            }
            const int src = SLLBM_CHK(eq ? 0 : ((kind == REC_BB || kind == REC_BB_ISO) ? C.opp[i] : i), Q, G.status, SLLBM_DEV_BAD_POP);
            const V2* p = fg + int64_t(src) * NN;
            if (D == 2) {
#pragma unroll
                for (int b = 0; b <= P; ++b)
#pragma unroll
                    for (int a = 0; a <= P; ++a) v[u][b * T1 + a] = __ldg(p + off[0][a] + off[1][b]);
            } else {
#pragma unroll
                for (int c3 = 0; c3 <= P; ++c3)
#pragma unroll
                    for (int b = 0; b <= P; ++b)
#pragma unroll
                        for (int a = 0; a <= P; ++a)
                            v[u][(c3 * T1 + b) * T1 + a] = __ldg(p + off[0][a] + off[1][b] + off[2][c3]);
            }
        }
#pragma unroll
        for (int u = 0; u < GV; ++u) {
            const int i = i0 + u;
            if (i >= Q) break;
            const int kind = (cw[u] >> 24) & 15;
            const int bid = (cw[u] >> 28) & 15;
            real of = 0, og = 0;
            if (kind == REC_EQ) {
                of = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                og = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            } else {
                if (D == 2) {
#pragma unroll
                    for (int b = 0; b <= P; ++b) {
                        real tf = 0, tg = 0;
#pragma unroll
                        for (int a = 0; a <= P; ++a) {
                            tf += wt[u][0][a] * v[u][b * T1 + a].x;
                            tg += wt[u][0][a] * v[u][b * T1 + a].y;
                        }
                        of += wt[u][1][b] * tf;
                        og += wt[u][1][b] * tg;
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
                                tf += wt[u][0][a] * v[u][(c3 * T1 + b) * T1 + a].x;
                                tg += wt[u][0][a] * v[u][(c3 * T1 + b) * T1 + a].y;
                            }
                            uf += wt[u][1][b] * tf;
                            ug += wt[u][1][b] * tg;
                        }
                        of += wt[u][2][c3] * uf;
                        og += wt[u][2][c3] * ug;
                    }
                }
                if (kind == REC_BB || kind == REC_BB_ISO) of += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
            }
            Sf[i * stride] = of;
            Sg[i * stride] = og;
        }
    }
    collide_smem<VSET, real, V2, 128>(C, Sf, Sg, twt[n], fgo + n, int(NN));
}

template <int VS, int P, typename real>
int launch_step_gather_smem(const StepLaunch<real>& L) {
    constexpr int Q = VelSet<VS>::Q;
    const int bs = 128;
    const int64_t grid = (L.G.n_nodes + bs - 1) / bs;
    const size_t smem = sizeof(real) * 2 * Q * bs;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_step_gather_smem<VS, P, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    k_step_gather_smem<VS, P, real><<<unsigned(grid), bs, smem, L.stream>>>(L.fg, L.fgo, L.code, L.gxi, L.tw, L.G,
                                                                          *L.C);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

template <int VS, int P, typename real>
int launch_step_structured(const StepLaunch<real>& L) {
    const int bs = 128;
    const int64_t grid = (L.G.n_nodes + bs - 1) / bs;
    k_step_structured<VS, P, real><<<unsigned(grid), bs, 0, L.stream>>>(L.fg, L.fgo, L.cls, L.tw, L.G, *L.C);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

template <int VS, int P, typename real>
int launch_step_structured_smem(const StepLaunch<real>& L) {
    constexpr int Q = VelSet<VS>::Q;
    const int bs = 128;
    const int64_t grid = (L.G.n_nodes + bs - 1) / bs;
    const size_t smem = sizeof(real) * 2 * Q * bs;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_step_structured_smem<VS, P, real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem));
    k_step_structured_smem<VS, P, real><<<unsigned(grid), bs, smem, L.stream>>>(L.fg, L.fgo, L.cls, L.tw, L.G,
                                                                              *L.C);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

template <int VS, int P, typename real>
int launch_step_gather(const StepLaunch<real>& L) {
    const int bs = 128;
    const int64_t grid = (L.G.n_nodes + bs - 1) / bs;
    k_step_gather<VS, P, real><<<unsigned(grid), bs, 0, L.stream>>>(L.fg, L.fgo, L.code, L.gxi, L.tw, L.G, *L.C,
                                                                     nullptr);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

#define SLLBM_EXTERN_STEP(VS, P, real)                                                   \
    extern template int launch_step_structured<VS, P, real>(const StepLaunch<real>&);    \
    extern template int launch_step_gather<VS, P, real>(const StepLaunch<real>&);        \
    extern template int launch_step_gather_smem<VS, P, real>(const StepLaunch<real>&);
#define SLLBM_EXTERN_TILED(VS, real)                                              \
    extern template int launch_step_tiled<VS, real, 0>(const StepLaunch<real>&);  \
    extern template int launch_step_tiled_smem<VS, real>(const StepLaunch<real>&);
#define SLLBM_INSTANTIATE_TILED(VS, real)                                  \
    template int launch_step_tiled<VS, real, 0>(const StepLaunch<real>&);  \
    template int launch_step_tiled_smem<VS, real>(const StepLaunch<real>&);
#define SLLBM_EXTERN_TILED_MLP(VS, real)                                          \
    extern template int launch_step_tiled<VS, real, 1>(const StepLaunch<real>&);  \
    extern template int launch_step_tiled<VS, real, 2>(const StepLaunch<real>&);  \
    extern template int launch_step_tiled_smem_tc<VS, real>(const StepLaunch<real>&);
#define SLLBM_INSTANTIATE_TILED_MLP(VS, real)                              \
    template int launch_step_tiled<VS, real, 1>(const StepLaunch<real>&);  \
    template int launch_step_tiled<VS, real, 2>(const StepLaunch<real>&);  \
    template int launch_step_tiled_smem_tc<VS, real>(const StepLaunch<real>&);

#define SLLBM_INSTANTIATE_STEP(VS, P, real)                                              \
    template int launch_step_structured<VS, P, real>(const StepLaunch<real>&);           \
    template int launch_step_gather<VS, P, real>(const StepLaunch<real>&);               \
    template int launch_step_gather_smem<VS, P, real>(const StepLaunch<real>&);
// orders whose fully unrolled kernels would be too large (3D, p = 4): the
// runtime-loop structured and gather kernels only
#define SLLBM_EXTERN_STEP_COMPACT(VS, P, real)                                                \
    extern template int launch_step_structured_smem<VS, P, real>(const StepLaunch<real>&);    \
    extern template int launch_step_gather_smem<VS, P, real>(const StepLaunch<real>&);
#define SLLBM_INSTANTIATE_STEP_COMPACT(VS, P, real)                                    \
    template int launch_step_structured_smem<VS, P, real>(const StepLaunch<real>&);    \
    template int launch_step_gather_smem<VS, P, real>(const StepLaunch<real>&);
#define SLLBM_ROW_WIDTHS(X, VS, real) X(VS, real, 32) X(VS, real, 64) X(VS, real, 128) X(VS, real, 192) X(VS, real, 256)
#define SLLBM_EXTERN_ROW1(VS, real, W) extern template int launch_step_row_smem<VS, real, W>(const StepLaunch<real>&);
#define SLLBM_INSTANTIATE_ROW1(VS, real, W) template int launch_step_row_smem<VS, real, W>(const StepLaunch<real>&);
#define SLLBM_EXTERN_ROW(VS, real) SLLBM_ROW_WIDTHS(SLLBM_EXTERN_ROW1, VS, real)
#define SLLBM_INSTANTIATE_ROW(VS, real) SLLBM_ROW_WIDTHS(SLLBM_INSTANTIATE_ROW1, VS, real)
// bulk-copy row kernel: widths whose six stages fit next to the state (D3Q45 up to 128 nodes)
#define SLLBM_ROWC_WIDTHS(X, VS, real) X(VS, real, 32) X(VS, real, 64) X(VS, real, 128) SLLBM_ROWC_W256_##VS(X, real)
#define SLLBM_ROWC_W256_1(X, real) X(1, real, 256)
#define SLLBM_ROWC_W256_3(X, real)
#define SLLBM_EXTERN_ROWC1(VS, real, W) extern template int launch_step_row_copy<VS, real, W, 6>(const StepLaunch<real>&);
#define SLLBM_INSTANTIATE_ROWC1(VS, real, W) template int launch_step_row_copy<VS, real, W, 6>(const StepLaunch<real>&);
#define SLLBM_EXTERN_ROWC(VS, real) SLLBM_ROWC_WIDTHS(SLLBM_EXTERN_ROWC1, VS, real)
#define SLLBM_INSTANTIATE_ROWC(VS, real) SLLBM_ROWC_WIDTHS(SLLBM_INSTANTIATE_ROWC1, VS, real)
#define SLLBM_ROWP_WIDTHS(X, VS, real) X(VS, real, 32) X(VS, real, 64) X(VS, real, 128) X(VS, real, 256)
#define SLLBM_EXTERN_ROWP1(VS, real, W) extern template int launch_step_row_p<VS, 4, real, W>(const StepLaunch<real>&);
#define SLLBM_INSTANTIATE_ROWP1(VS, real, W) template int launch_step_row_p<VS, 4, real, W>(const StepLaunch<real>&);
#define SLLBM_EXTERN_ROWP(VS, real) SLLBM_ROWP_WIDTHS(SLLBM_EXTERN_ROWP1, VS, real)
#define SLLBM_INSTANTIATE_ROWP(VS, real) SLLBM_ROWP_WIDTHS(SLLBM_INSTANTIATE_ROWP1, VS, real)
#define SLLBM_EXTERN_TILED_P(VS, P, real) extern template int launch_step_tiled_p<VS, P, real>(const StepLaunch<real>&);
#define SLLBM_INSTANTIATE_TILED_P(VS, P, real) template int launch_step_tiled_p<VS, P, real>(const StepLaunch<real>&);

}  // namespace sllbm
