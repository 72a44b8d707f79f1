// C ABI of the SLLBM library: context lifecycle, setup orchestration, step
// dispatch and readouts.  See include/sllbm.h for the contract of each call.
#include <algorithm>
#include <cmath>
#include <limits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "sllbm_internal.h"
#include "mlp.cuh"
#include "step_kernels.cuh"

namespace sllbm {
int launch_trace(const TraceArgs& A, const double* dX, int64_t n_units, int structured, int ncls0, int ncls1,
                 Rec64* out, int* d_fail, cudaStream_t s);
int launch_isothermal(const Rec64* rec, int64_t n_units, int Q, const double* bcT, double* Tw,
                      unsigned long long* counts, cudaStream_t s);
template <typename real>
int launch_pack_gather(const Rec64* rec, int64_t N, int Q, int D, int32_t* code, real* xi, cudaStream_t s);
template <typename real>
int launch_init(int vs, const double* rho, const double* u, const double* T, int64_t N, const CollideConst<double>& C,
                typename Vec2<real>::T* fg, cudaStream_t s);
template <typename real>
int launch_convert(typename Vec2<real>::T* fgd, double* ff, double* gf, int64_t N, int Q, const double* w,
                   const double* wg, int dir, cudaStream_t s);
template <typename real>
int launch_moments(int vs, const typename Vec2<real>::T* fg, int64_t N, const CollideConst<double>& C, double* rho,
                   double* u, double* T, cudaStream_t s);
template <typename real>
int launch_conserve(int vs, int D, const typename Vec2<real>::T* fg, int64_t N, const CollideConst<double>& C,
                    double* part, int* flag, double* out, cudaStream_t s);
int conserve_blocks();
void k_reduce_parts_launch(const double* part, int nblk, int K, double* out, cudaStream_t s);
template <typename real>
int launch_step_generic(int p, int D, const StepLaunch<real>& L, const GenVel<real>* V, int Q);
template <typename real>
int launch_init_generic(const double* rho, const double* u, const double* T, int64_t N, const GenVel<double>* V,
                        int Q, int D, typename Vec2<real>::T* fg, cudaStream_t s);
template <typename real>
int launch_moments_generic(const typename Vec2<real>::T* fg, int64_t N, const GenVel<double>* V, int Q, int D,
                           double cv, double* rho, double* u, double* T, cudaStream_t s);
template <typename real>
int launch_conserve_generic(const typename Vec2<real>::T* fg, int64_t N, const GenVel<double>* V, int Q, int D,
                            double cv, int grid_stride, unsigned blocks, double* part, int* flag, cudaStream_t s);
template <typename V2>
int launch_x_layers(V2* fg, V2* buf, int64_t NN, int Nx, int rows, int x0, int nx, int Q, int dir, cudaStream_t s);
template <typename real>
int launch_scale_state(typename Vec2<real>::T* fg, int64_t N, int Q, const double* w, const double* wg, double s,
                       cudaStream_t st);
SLLBM_EXTERN_STEP(0, 2, float)
SLLBM_EXTERN_STEP(1, 2, float)
SLLBM_EXTERN_STEP(1, 3, float)
SLLBM_EXTERN_STEP(2, 2, float)
SLLBM_EXTERN_STEP(3, 2, float)
SLLBM_EXTERN_STEP(0, 2, double)
SLLBM_EXTERN_STEP(1, 2, double)
SLLBM_EXTERN_STEP(1, 3, double)
SLLBM_EXTERN_STEP(2, 2, double)
SLLBM_EXTERN_STEP(3, 2, double)
SLLBM_EXTERN_STEP(0, 4, float)
SLLBM_EXTERN_STEP(1, 4, float)
SLLBM_EXTERN_STEP(2, 4, float)
SLLBM_EXTERN_STEP_COMPACT(3, 4, float)
SLLBM_EXTERN_STEP(0, 4, double)
SLLBM_EXTERN_STEP(1, 4, double)
SLLBM_EXTERN_STEP(2, 4, double)
SLLBM_EXTERN_STEP_COMPACT(3, 4, double)
SLLBM_EXTERN_ROWP(1, float)
SLLBM_EXTERN_ROWP(3, float)
SLLBM_EXTERN_ROW(1, float)
SLLBM_EXTERN_ROW(3, float)
SLLBM_EXTERN_ROWC(1, float)
SLLBM_EXTERN_ROWC(3, float)
SLLBM_EXTERN_TILED_P(0, 4, float)
SLLBM_EXTERN_TILED_P(1, 4, float)
SLLBM_EXTERN_TILED_P(2, 4, float)
SLLBM_EXTERN_TILED_P(3, 4, float)
SLLBM_EXTERN_TILED_P(0, 4, double)
SLLBM_EXTERN_TILED_P(1, 4, double)
SLLBM_EXTERN_TILED_P(2, 4, double)
SLLBM_EXTERN_TILED_P(3, 4, double)
SLLBM_EXTERN_TILED(0, float)
SLLBM_EXTERN_TILED(1, float)
SLLBM_EXTERN_TILED(2, float)
SLLBM_EXTERN_TILED(3, float)
SLLBM_EXTERN_TILED(0, double)
SLLBM_EXTERN_TILED(1, double)
SLLBM_EXTERN_TILED(2, double)
SLLBM_EXTERN_TILED(3, double)
SLLBM_EXTERN_TILED_MLP(1, float)
int launch_moments_f32(int vs, const float2* fg, int64_t N, const CollideConst<float>& C, double cv, double* rho,
                       double* u, double* T, cudaStream_t s);
int plane_stat_count(int D);
int launch_plane_sums(const double* rho, const double* u, const double* T, int D, int N0, int N1, int N2,
                      double* out, int accumulate, cudaStream_t s);
int launch_plane_cp(const double* rho, const double* T, int N0, int N1, int N2, int j, double p0, double denom,
                    double* out, cudaStream_t s);
void build_moment_basis(const HostVelSet& vs, std::vector<double>& Phi, std::vector<double>& Ginv,
                        std::vector<double>& P);
bool rows_tmem_shape(int D, int nx, int& ty, int& tz);
bool rows_pairs_shape(int D, int nx, int p, int& ty, int& tz);
int launch_rows_pairs(int vs, int nx, const float2* fg, float2* fgo, const void* maps, const int32_t* head,
                      const void* recs, const uint64_t* xmask, const uint64_t* smask, const float* tw,
                      const StepGeom& G, const CollideConst<float>& C, const TmGeom2& T, int* status, cudaStream_t s,
                      int grid);
size_t rows_tmem_smem_bytes(int D, int nx, const TmGeom& T);
int launch_rows_tmem(int vs, int nx, const float2* fg, float2* fgo, const float* bop, const int32_t* head,
                     const TmRec* recs, const uint64_t* xmask, const float* tw, const StepGeom& G,
                     const CollideConst<float>& C, const TmGeom& T, int* status, cudaStream_t s, int grid);
void build_moment_basis(const HostVelSet& vs, std::vector<double>& Phi, std::vector<double>& Ginv,
                        std::vector<double>& P, std::vector<int>* degree);
}  // namespace sllbm

using namespace sllbm;

namespace {

thread_local std::string g_create_error;

int fail(sllbm_ctx* c, int code, const std::string& msg) {
    if (c) c->last_error = msg; else g_create_error = msg;
    return code;
}

int cuda_fail(sllbm_ctx* c, cudaError_t e, const char* what) {
    if (c && c->bad_alloc) {
        c->bad_alloc = false;
        return fail(c, SLLBM_ERR_ARG,
                    std::string(what) + ": the allocator returned memory that is not 256-byte aligned device "
                                        "memory of the context's GPU");
    }
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? SLLBM_ERR_NOMEM : SLLBM_ERR_CUDA, m);
}

// Device memory of a context: from the caller's allocator when one was set
// (sllbm_set_allocator) at the context's creation, else cudaMalloc / cudaFree.
// The caller's memory must be device memory of the context's GPU, 256-byte
// aligned; anything else is handed back and reported.
cudaError_t dev_alloc(sllbm_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (!c->alloc_fn) return cudaMalloc(p, bytes);
    void* q = c->alloc_fn(bytes, c->alloc_user);
    if (!q) return cudaErrorMemoryAllocation;
    cudaPointerAttributes at{};
    const bool ok = (reinterpret_cast<uintptr_t>(q) % 256) == 0 && cudaPointerGetAttributes(&at, q) == cudaSuccess &&
                    at.type == cudaMemoryTypeDevice && at.device == c->device;
    if (!ok) {
        cudaGetLastError();
        c->free_fn(q, c->alloc_user);
        c->bad_alloc = true;
        return cudaErrorInvalidValue;
    }
    *p = q;
    return cudaSuccess;
}
void dev_free(sllbm_ctx* c, void* p) {
    if (!p) return;
    if (c->alloc_fn)
        c->free_fn(p, c->alloc_user);
    else
        cudaFree(p);
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

size_t real_size(const sllbm_ctx* c) { return c->precision == SLLBM_FP64 ? 8 : 4; }

// host evaluation of the equilibrium deviations (same scalar polynomial as the kernels)
void host_eq_dev(const sllbm_ctx* c, double rho, const double* u, double T, double* fdev, double* gdev) {
    const HostVelSet& vs = c->vs;
    const int D = vs.D;
    const double cv = 1.0 / (c->params.gamma - 1.0);
    const double gf = 2.0 * cv - D;
    double U = 0;
    for (int d = 0; d < D; ++d) U += u[d] * u[d];
    const double t = T - 1.0;
    for (int i = 0; i < vs.Q; ++i) {
        double s = 0, cd = 0;
        for (int d = 0; d < D; ++d) {
            s += vs.xi[i * D + d] * vs.xi[i * D + d];
            cd += vs.xi[i * D + d] * u[d];
        }
        const double A = s - D, B = s - D - 2, Cc = s - D - 4, E = s * s - 2.0 * (D + 2) * s + D * (D + 2.0);
        const double k2 = 0.5 - 0.25 * U + 0.25 * t * Cc;
        const double k1 = 1.0 - 0.5 * U + 0.5 * t * B;
        const double k0 = -0.5 * U + 0.125 * U * U + 0.5 * t * A - 0.25 * t * U * B + 0.125 * t * t * E;
        const double P1 = (((cd / 24.0 + 1.0 / 6.0) * cd + k2) * cd + k1) * cd + k0;
        fdev[i] = vs.w[i] * (rho * P1 + (rho - 1.0));
        gdev[i] = vs.w[i] * gf * (rho * T * P1 + (rho * T - 1.0));
    }
}

template <typename real>
void fill_collide_const(sllbm_ctx* c, CollideConst<real>& C) {
    std::memset(&C, 0, sizeof(C));
    const HostVelSet& vs = c->vs;
    const int D = vs.D;
    const double cv = 1.0 / (c->params.gamma - 1.0);
    const double gf = 2.0 * cv - D;
    // the per-velocity arrays hold the compiled sets (Q <= SLLBM_QMAX); the
    // generic sets keep theirs in the GenVel table
    const int Qc = std::min(vs.Q, SLLBM_QMAX);
    for (int i = 0; i < Qc; ++i) {
        for (int d = 0; d < D; ++d) C.xi[i][d] = real(vs.xi[i * D + d]);
        C.w[i] = real(vs.w[i]);
        C.wg[i] = real(vs.w[i] * gf);
        C.opp[i] = vs.opp[i];
        double s = 0;
        for (int d = 0; d < D; ++d) s += vs.xi[i * D + d] * vs.xi[i * D + d];
        C.s2v[i] = real(s);
        C.sAv[i] = real(s - D);
        C.sBv[i] = real(s - D - 2);
        C.sCv[i] = real(s - D - 4);
        C.sEv[i] = real(s * s - 2.0 * (D + 2) * s + D * (D + 2.0));
        static const int xa[6] = {0, 1, 2, 0, 0, 1}, xb[6] = {0, 1, 2, 1, 2, 2};
        for (int k = 0; k < 6; ++k)
            C.xx[i][k] = xa[k] < D && xb[k] < D ? real(vs.xi[i * D + xa[k]] * vs.xi[i * D + xb[k]]) : real(0);
    }
    for (size_t h = 0; h < vs.shell_s.size(); ++h) {
        const double s = vs.shell_s[h];
        C.sA[h] = real(s - D);
        C.sB[h] = real(s - D - 2);
        C.sC[h] = real(s - D - 4);
        C.sE[h] = real(s * s - 2.0 * (D + 2) * s + D * (D + 2.0));
        C.s2[h] = real(s);
    }
    C.cv = real(cv);
    C.gfac = real(gf);
    C.dt = real(c->params.dt);
    C.inv_Pr = real(1.0 / c->params.Pr);
    C.mu_ref = real(c->params.mu_ref);
    C.inv_T_ref = real(1.0 / c->params.T_ref);
    C.mu_exp = real(c->params.mu_exp);
    C.var_mu = c->params.mu_exp != 0.0;
    C.quasi = c->params.Pr != 1.0;
    C.forced = (c->force[0] != 0.0 || c->force[1] != 0.0 || c->force[2] != 0.0) ? 1 : 0;
    for (int d = 0; d < 3; ++d) C.force_dt[d] = real(d < D ? c->force[d] * c->params.dt : 0.0);
    for (int b = 0; b < 2; ++b) {
        const sllbm_bc& bc = c->desc.bc[b];
        std::vector<double> fe(vs.Q), ge(vs.Q);
        host_eq_dev(c, bc.rho, bc.u, bc.T, fe.data(), ge.data());
        for (int i = 0; i < Qc; ++i) {
            C.eqf[b][i] = real(fe[i]);
            C.eqg[b][i] = real(ge[i]);
            double cu = 0;
            for (int d = 0; d < D; ++d) cu += vs.xi[i * D + d] * bc.u[d];
            C.mw[b][i] = real(2.0 * vs.w[i] * bc.rho * cu);
        }
    }
}

// The generic kernels' per-velocity table (GenVel): the quantities
// fill_collide_const puts in CollideConst's per-velocity arrays, for any Q.
template <typename real>
void build_gen_table(const sllbm_ctx* c, std::vector<GenVel<real>>& out) {
    const HostVelSet& vs = c->vs;
    const int D = vs.D, Q = vs.Q;
    const double cv = 1.0 / (c->params.gamma - 1.0);
    const double gf = 2.0 * cv - D;
    out.assign(Q, GenVel<real>{});
    std::vector<double> fe[2], ge[2];
    for (int b = 0; b < 2; ++b) {
        fe[b].resize(Q);
        ge[b].resize(Q);
        const sllbm_bc& bc = c->desc.bc[b];
        host_eq_dev(c, bc.rho, bc.u, bc.T, fe[b].data(), ge[b].data());
    }
    for (int i = 0; i < Q; ++i) {
        GenVel<real>& v = out[i];
        double s = 0;
        for (int d = 0; d < D; ++d) {
            v.xi[d] = real(vs.xi[i * D + d]);
            s += vs.xi[i * D + d] * vs.xi[i * D + d];
        }
        v.w = real(vs.w[i]);
        v.wg = real(vs.w[i] * gf);
        v.s2 = real(s);
        v.sA = real(s - D);
        v.sB = real(s - D - 2);
        v.sC = real(s - D - 4);
        v.sE = real(s * s - 2.0 * (D + 2) * s + D * (D + 2.0));
        for (int b = 0; b < 2; ++b) {
            const sllbm_bc& bc = c->desc.bc[b];
            v.eqf[b] = real(fe[b][i]);
            v.eqg[b] = real(ge[b][i]);
            double cu = 0;
            for (int d = 0; d < D; ++d) cu += vs.xi[i * D + d] * bc.u[d];
            v.mw[b] = real(2.0 * vs.w[i] * bc.rho * cu);
        }
        v.opp = vs.opp[i];
    }
}

template <typename real>
void build_class_table(const sllbm_ctx* c, const std::vector<Rec64>& rec, std::vector<ClassRec<real>>& out) {
    const HostMesh& m = c->mesh;
    const int Q = c->vs.Q, D = m.D, p = m.p;
    const int64_t U = c->n_rec_units;
    out.assign(size_t(Q * U), ClassRec<real>());
    for (int i = 0; i < Q; ++i)
        for (int64_t u = 0; u < U; ++u) {
            const Rec64& r = rec[size_t(i * U + u)];
            ClassRec<real>& o = out[size_t(i * U + u)];
            std::memset(&o, 0, sizeof(o));
            o.meta = r.meta;
            if (r.cell < 0) continue;
            int cc[3] = {0, 0, 0};
            int64_t cl = r.cell;
            for (int d = 0; d < D; ++d) {
                cc[d] = int(cl % m.cells[d]);
                cl /= m.cells[d];
            }
            for (int d = 0; d < D; ++d) {
                o.cell[d] = cc[d];   // periodic dims: representative home cell is 0 -> offset
                for (int a = 0; a <= p; ++a) {
                    double v = 1.0;
                    for (int q = 0; q <= p; ++q)
                        if (q != a) v *= (r.xi[d] - m.glc[q]) / (m.glc[a] - m.glc[q]);
                    o.wt[d][a] = real(v);
                }
            }
        }
}

// Builds the constant part of the learned-collision image (moment basis,
// inverse Gram matrix) on first use; weights arrive with sllbm_mlp_set.
int ensure_mlp_image(sllbm_ctx* ctx) {
    if (ctx->mlp_img) return SLLBM_OK;
    if (ctx->precision != SLLBM_FP32 || !(ctx->tiled && ctx->velset == SLLBM_D2Q19))
        return fail(ctx, SLLBM_ERR_UNSUPPORTED,
                    "learned collision is built for FP32 D2Q19 contexts with the warp-tiled structured kernel");
    const int Q = ctx->vs.Q, D = ctx->vs.D;
    std::vector<double> Phi, Ginv, P;
    build_moment_basis(ctx->vs, Phi, Ginv, P);
    const int n = mlp_image_floats(Q, D);
    std::vector<float> img(n, 0.0f);
    const int H = MLP_H;
    const int o_sin = H * Q + H * H + Q * H + 2 * H + Q;
    const int o_phi = o_sin + Q;
    const int o_gi = o_phi + Q * Q;
    for (int k = 0; k < Q * Q; ++k) img[o_phi + k] = float(Phi[k]);
    for (int k = 0; k < (D + 2) * (D + 2); ++k) img[o_gi + k] = float(Ginv[k]);
    img[n - 1] = 1.0f;
    ctx->mlp_host = img;
    CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->mlp_img), sizeof(float) * n));
    CK(cudaMemcpyAsync(ctx->mlp_img, img.data(), sizeof(float) * n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SLLBM_OK;
}

// Warp-tiled records: per (velocity, class) the (y, z) source-row offsets
// relative to the arrival node (no periodic wrap; the kernel recomputes them
// near a seam from the packed dy / dz), the weight products and the x taps as
// lane offsets.
template <typename real>
void build_tile_table(const sllbm_ctx* c, const std::vector<Rec64>& rec, std::vector<TileRec<real>>& out) {
    const HostMesh& m = c->mesh;
    const StepGeom& G = c->geom;
    const int Q = c->vs.Q, D = m.D;
    const int64_t U = c->n_rec_units;
    out.assign(size_t(Q * U), TileRec<real>());
    const int Nx = m.N[0], N1 = m.N[1];
    for (int i = 0; i < Q; ++i)
        for (int64_t u = 0; u < U; ++u) {
            const Rec64& r = rec[size_t(i * U + u)];
            TileRec<real>& o = out[size_t(i * U + u)];
            std::memset(&o, 0, sizeof(o));
            o.meta = r.meta;
            if (r.cell < 0) continue;
            // representative node of the class
            const int k0 = int(u % G.ncls[0]);
            const int k1 = int((u / G.ncls[0]) % G.ncls[1]);
            const int k2 = int(u / (int64_t(G.ncls[0]) * G.ncls[1]));
            const int cc0 = int(r.cell % m.cells[0]);
            const int cc1 = int((r.cell / m.cells[0]) % m.cells[1]);
            const int cc2 = int(r.cell / (int64_t(m.cells[0]) * m.cells[1]));
            double L[3][3];
            for (int d = 0; d < D; ++d)
                for (int a = 0; a <= 2; ++a) {
                    double v = 1.0;
                    for (int q = 0; q <= 2; ++q)
                        if (q != a) v *= (r.xi[d] - m.glc[q]) / (m.glc[a] - m.glc[q]);
                    L[d][a] = v;
                }
            int dx[3], dy[3], dz[3] = {0, 0, 0};
            for (int a = 0; a <= 2; ++a) {
                int d = cc0 * 2 + a - k0;
                if (d > Nx / 2) d -= Nx;
                if (d < -Nx / 2) d += Nx;
                dx[a] = d;
                dy[a] = cc1 * 2 + a - k1;     // periodic y: offsets from the representative (home cell 0)
                if (m.periodic[1]) {
                    if (dy[a] > N1 / 2) dy[a] -= N1;
                    if (dy[a] < -N1 / 2) dy[a] += N1;
                }
                if (D == 3) {
                    dz[a] = cc2 * 2 + a - k2;
                    if (dz[a] > m.N[2] / 2) dz[a] -= m.N[2];
                    if (dz[a] < -m.N[2] / 2) dz[a] += m.N[2];
                }
            }
            o.dxp = (dx[0] + 8) | ((dx[1] + 8) << 4) | ((dx[2] + 8) << 8);
            o.dyzp = (dy[0] + 8) | ((dy[1] + 8) << 4) | ((dy[2] + 8) << 8) | ((dz[0] + 8) << 12) |
                     ((dz[1] + 8) << 16) | ((dz[2] + 8) << 20);
            const int NR = D == 3 ? 9 : 3;
            for (int k = 0; k < NR; ++k) {
                const int b = k % 3, cz = k / 3;
                o.rel[k] = dy[b] * Nx + (D == 3 ? dz[cz] * Nx * N1 : 0);
                o.rw[k] = real(L[1][b] * (D == 3 ? L[2][cz] : 1.0));
            }
            for (int a = 0; a <= 2; ++a) o.wx[a] = real(L[0][a]);
        }
}

// True when, for every velocity and every (y, z) class, the records of the two
// x parities share kind, source population, y/z offsets and y/z weights: the
// source rows of a velocity are then the same for a whole periodic x row.
template <typename real>
bool row_uniform_table(const sllbm_ctx* c, const std::vector<TileRec<real>>& t) {
    const StepGeom& G = c->geom;
    if (G.ncls[0] != 2) return false;
    for (int i = 0; i < c->vs.Q; ++i)
        for (int cl = 0; cl < G.n_classes; cl += 2) {
            const TileRec<real>& a = t[size_t(i) * G.n_classes + cl];
            const TileRec<real>& b = t[size_t(i) * G.n_classes + cl + 1];
            if (a.meta != b.meta || a.dyzp != b.dyzp) return false;
            for (int k = 0; k < 9; ++k)
                if (a.rw[k] != b.rw[k]) return false;
        }
    return true;
}

// Tables of the tensor-memory row-tile kernel (step_tmem.cuh) from the warp
// tile records: tiles of TY x TZ whole x rows.  Per (velocity, tile class):
// the source rows that the (y, z) taps of the tile's rows read -- taps of
// zero weight dropped (a velocity with no motion along an axis interpolates
// at a node: one tap there) -- as runs of consecutive y rows per (population,
// z), each run one contiguous block of memory (one bulk copy; rows between
// two needed ones are copied too); per (row, x parity) the record with the
// taps' row slots in the stage; per tile class the velocities whose x factor
// is not the identity.  Returns false (tables not built) where the kernel
// does not apply.
// FP32 rounded to TF32 (10 mantissa bits, nearest, ties away from zero: the
// device's cvt.rna.tf32.f32)
float tf32_rna(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    float o;
    std::memcpy(&o, &u, 4);
    return o;
}

// byte offset of element (r, k) of an R x K FP32/TF32 operand in the
// canonical K-major layout without swizzle: 8 x 16-byte core matrices, 128 B
// apart along K and K * 32 B apart along R (K a multiple of 4)
inline int tf32_canon_offset(int r, int k, int K) {
    return (r >> 3) * (K * 32) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

bool build_rows_tmem(sllbm_ctx* c, const std::vector<TileRec<float>>& t, std::vector<int32_t>& head,
                     std::vector<TmRec>& recs, std::vector<uint64_t>& xmask, std::vector<float>& bop) {
    const HostMesh& m = c->mesh;
    const StepGeom& G = c->geom;
    const int Q = c->vs.Q, D = m.D, NX = m.N[0], N1 = m.N[1], N2 = D == 3 ? m.N[2] : 1;
    int TY = 0, TZ = 0;
    if (c->precision != SLLBM_FP32 || m.p != 2 || !c->tiled || !c->row_uniform) return false;
    if (!((c->velset == SLLBM_D3Q45 && D == 3) || (c->velset == SLLBM_D2Q19 && D == 2))) return false;
    if (!rows_tmem_shape(D, NX, TY, TZ) || G.ncls[0] != 2 || !m.periodic[0]) return false;
    const bool py = m.periodic[1] != 0;
    if (py && N1 % TY) return false;
    if (D == 3 && (!m.periodic[2] || N2 % TZ)) return false;
    if (int64_t(Q) * m.n_nodes >= (int64_t(1) << 31)) return false;
    const int NR = TY * TZ;
    TmGeom T{};
    T.ntile_y = (N1 + TY - 1) / TY;
    T.ntile_z = D == 3 ? N2 / TZ : 1;
    T.ntiles = T.ntile_y * T.ntile_z;
    T.n_tc = py ? 1 : T.ntile_y;
    head.assign(size_t(Q) * T.n_tc * TM_HEAD, 0);
    recs.assign(size_t(Q) * T.n_tc * NR * 2, TmRec{});
    xmask.assign(size_t(T.n_tc), 0);
    const int NRT = D == 3 ? 9 : 3;
    int max_rows = 1;
    struct Tap {
        int src, dy, dz;
        float w;
    };
    for (int i = 0; i < Q; ++i)
        for (int tc = 0; tc < T.n_tc; ++tc) {
            const int y0 = py ? 0 : tc * TY;
            int32_t* h = &head[(size_t(i) * T.n_tc + tc) * TM_HEAD];
            std::vector<std::vector<Tap>> taps(NR);     // per row of the tile
            std::vector<int> cls0(NR, -1);
            for (int r = 0; r < NR; ++r) {
                const int ry = r % TY, rz = r / TY;
                const int y = y0 + ry, z = rz;
                if (y >= N1) continue;                   // beyond a ragged last tile: an idle row
                cls0[r] = G.ncls[0] * ((py ? (y & 1) : y) + G.ncls[1] * (D == 3 ? (z & 1) : 0));
                const TileRec<float>& a = t[size_t(i) * G.n_classes + cls0[r]];
                if ((a.meta & 15) == REC_EQ) continue;
                for (int k = 0; k < NRT; ++k) {
                    const float wk = a.rw[k];
                    if (std::fabs(wk) < 1e-12f) continue;
                    const int dy = ((a.dyzp >> (4 * (k % 3))) & 15) - 8;
                    const int dz = D == 3 ? ((a.dyzp >> (12 + 4 * (k / 3))) & 15) - 8 : 0;
                    taps[r].push_back({a.meta >> 8, ry + dy, rz + dz, wk});
                }
            }
            // runs: per (population, z) the y range from the lowest to the highest row read
            struct Run {
                int src, dz, ylo, yhi, slot;
            };
            std::vector<Run> runs;
            for (int r = 0; r < NR; ++r)
                for (const Tap& tp : taps[r]) {
                    bool found = false;
                    for (Run& u : runs)
                        if (u.src == tp.src && u.dz == tp.dz) {
                            u.ylo = std::min(u.ylo, tp.dy);
                            u.yhi = std::max(u.yhi, tp.dy);
                            found = true;
                        }
                    if (!found) runs.push_back({tp.src, tp.dz, tp.dy, tp.dy, 0});
                }
            if (int(runs.size()) > TM_MAX_RUNS) return false;
            int nrows = 0;
            for (size_t q = 0; q < runs.size(); ++q) {
                Run& u = runs[q];
                if (u.ylo + 128 < 0 || u.yhi + 128 > 255 || u.dz + 128 < 0 || u.dz + 128 > 255 ||
                    u.yhi - u.ylo + 1 > 63)
                    return false;
                u.slot = nrows;
                nrows += u.yhi - u.ylo + 1;
                h[2 + q] = tm_pack_run(u.src, u.ylo, u.dz, u.yhi - u.ylo + 1);
                h[2 + TM_MAX_RUNS + q] = u.slot;
            }
            if (nrows > TM_MAX_ROWS) return false;
            h[0] = int(runs.size());
            h[1] = nrows;
            max_rows = std::max(max_rows, nrows);
            bool xchg = false;
            for (int r = 0; r < NR; ++r) {
                TmRec* o = &recs[((size_t(i) * T.n_tc + tc) * NR + r) * 2];
                if (cls0[r] < 0) {
                    for (int xp = 0; xp < 2; ++xp) o[xp].meta = REC_EQ;
                    continue;
                }
                const TileRec<float>& a = t[size_t(i) * G.n_classes + cls0[r]];
                const int kind = a.meta & 15;
                for (int xp = 0; xp < 2; ++xp) {
                    const TileRec<float>& b = t[size_t(i) * G.n_classes + cls0[r] + xp];
                    if (b.meta != a.meta) return false;
                    TmRec& ro = o[xp];
                    ro.meta = b.meta;
                    ro.ntap = int(taps[r].size());
                    if (kind == REC_EQ) continue;
                    const int dx0 = (b.dxp & 15) - 8;
                    for (int q = 0; q < 3; ++q)
                        if (((b.dxp >> (4 * q)) & 15) - 8 != dx0 + q) return false;
                    if (dx0 < -2 || dx0 > 0) return false;
                    ro.dx0 = dx0;
                    for (int q = 0; q < 3; ++q) ro.wx[q] = b.wx[q];
                    for (size_t q = 0; q < taps[r].size(); ++q) {
                        const Tap& tp = taps[r][q];
                        int sl = -1;
                        for (const Run& u : runs)
                            if (u.src == tp.src && u.dz == tp.dz) sl = u.slot + tp.dy - u.ylo;
                        ro.off[q] = sl * NX * 8;
                        ro.w[q] = tp.w;
                    }
                    // the identity x factor: weight one at the node itself
                    bool ident = true;
                    for (int q = 0; q < 3; ++q) {
                        const double target = (dx0 + q == 0) ? 1.0 : 0.0;
                        if (std::fabs(double(b.wx[q]) - target) > 1e-12) ident = false;
                    }
                    if (!ident) xchg = true;
                }
            }
            if (xchg) xmask[tc] |= uint64_t(1) << i;
        }
    T.rows_bytes = max_rows * NX * 8;
    T.stage_bytes = T.rows_bytes + NR * 2 * int(sizeof(TmRec));
    size_t fixed = sizeof(float2) * 2 * NR * (NX + 4) + 16;
    if (c->want_tc) {
        // tensor-core variant (128-node rows, tiles of 4 rows): per (velocity,
        // tile class) the weights of the (y, z) contraction as the product's
        // B operand, N = 16 (rows of the tile, zero padded) x K = kp (the
        // velocity's source rows, zero padded), split into TF32 hi and lo
        // parts, in the canonical K-major layout
        if (NX != 128 || NR > 16) return false;
        const int kp = (max_rows + 7) / 8 * 8;
        T.kp = kp;
        bop.assign(size_t(Q) * T.n_tc * 2 * 16 * kp, 0.f);
        for (int i = 0; i < Q; ++i)
            for (int tc = 0; tc < T.n_tc; ++tc) {
                float* hi = &bop[(size_t(i) * T.n_tc + tc) * 2 * 16 * kp];
                float* lo = hi + 16 * kp;
                for (int r = 0; r < NR; ++r)
                    for (int xp = 0; xp < 1; ++xp) {
                        const TmRec& ro = recs[((size_t(i) * T.n_tc + tc) * NR + r) * 2 + xp];
                        if ((ro.meta & 15) == REC_EQ) continue;
                        for (int q = 0; q < ro.ntap; ++q) {
                            const int k = ro.off[q] / (NX * 8);
                            const float h = tf32_rna(ro.w[q]);
                            hi[tf32_canon_offset(r, k, kp) / 4] = h;
                            lo[tf32_canon_offset(r, k, kp) / 4] = tf32_rna(ro.w[q] - h);
                        }
                    }
            }
        T.stage_bytes += 2 * 16 * kp * 4;
        fixed += 4 * size_t(NX) * kp * 4 + 1024 + 8;       // the A operands (f, g x hi, lo), alignment, barrier
    }
    const size_t budget = 227 * 1024;
    int nst = int((budget - fixed) / (size_t(T.stage_bytes) + 16));
    nst = std::min(nst, 16) & ~1;         // a multiple of the two producer warps
    if (nst < 2) return false;
    T.nst = nst;
    c->tm = T;
    c->tm_ty = TY;
    c->tm_tz = TZ;
    return true;
}

// The stages of the two-nodes-per-thread kernel (both orders): two rings (one
// per consumer group) of two stages (one where the largest velocity needs
// more room) of `cap` rows and the records of up to
// maxv <= TM2_MAX_VEL velocities (measured on the channel: two large stages
// per ring beat three smaller ones); each group's velocities (i = h, h + 2, ...) are
// packed into stages per tile class, consecutive velocities while their rows
// fit `cap`; a velocity's slots and its records' tap offsets move by the rows
// before it.  Sets the kernel geometry; false where the stages do not fit.
template <class REC>
bool pack_rows_pairs(sllbm_ctx* c, TmGeom2& T, int NX, int NR, int max_rows, const std::vector<int>& shapes,
                     std::vector<int32_t>& head, std::vector<REC>& recs, std::vector<uint64_t>& smask) {
    const int Q = c->vs.Q;
    const int rec_bytes = NR * int(sizeof(REC));               // one velocity's records, as copied
    const int rec_slot = (rec_bytes + 127) / 128 * 128;        // their 128-byte aligned slot in a stage
    const size_t fixed = sizeof(float2) * 4 * NR * NX + 8 + 16;     // two exchange rows per group and row
    // all of an SM's shared memory for a 512-node tile (one CTA per SM), half
    // of it for a 256-node tile (two CTAs per SM)
    const size_t budget = NX * NR == 512 ? 227 * 1024 : 112 * 1024;
    // two stages per ring where the largest velocity's rows fit, else one;
    // the most velocities per stage whose records leave room for those rows
    int cap = 0, nst = 0, maxv = 0;
    for (int n : {4, 2}) {
        for (int v = TM2_MAX_VEL; v >= 1 && !maxv; --v) {
            const long long room = (static_cast<long long>(budget) - static_cast<long long>(fixed)) / n - 16 -
                                   static_cast<long long>(v) * rec_slot;
            const int k = int(std::max(0LL, room) / (NX * 8));
            if (k >= max_rows) {
                cap = k;
                maxv = v;
                nst = n;
            }
        }
        if (maxv) break;
    }
    if (!maxv) return false;
    smask.assign(size_t(2) * T.n_tc, 0);
    for (int tc = 0; tc < T.n_tc; ++tc)
        for (int hg = 0; hg < 2; ++hg) {
            const int nv = (Q - hg + 1) / 2;
            int j0 = 0;
            while (j0 < nv) {
                int rows = 0, n = 0;
                while (j0 + n < nv && n < maxv) {
                    const int i = hg + 2 * (j0 + n);
                    const int r_i = head[(size_t(i) * T.n_tc + tc) * TM2_HEAD + 1];
                    if (rows + r_i > cap) break;
                    rows += r_i;
                    ++n;
                }
                if (n == 0) return false;
                smask[size_t(tc) * 2 + hg] |= uint64_t(1) << j0;
                int base = 0;
                for (int q = 0; q < n; ++q) {
                    const int i = hg + 2 * (j0 + q);
                    int32_t* h = &head[(size_t(i) * T.n_tc + tc) * TM2_HEAD];
                    for (int b = 0; b < h[0]; ++b) h[2 + TM2_MAX_BOXES + b] += base;
                    for (int r = 0; r < NR; ++r) {
                        REC& ro = recs[(size_t(i) * T.n_tc + tc) * NR + r];
                        if ((ro.meta & 15) == REC_EQ) continue;
                        for (int k = 0; k < ro.ntap; ++k) ro.off[k] += base * NX * 8;
                    }
                    base += h[1];
                }
                int32_t* h0 = &head[(size_t(hg + 2 * j0) * T.n_tc + tc) * TM2_HEAD];
                h0[14] = 1 | (n << 8);
                h0[15] = rows * NX * 8 + n * rec_bytes;
                j0 += n;
            }
        }
    T.rows_bytes = cap * NX * 8;
    T.stage_bytes = T.rows_bytes + maxv * rec_slot;
    // every tensor copy's destination (stage, row block, records slot) 128-byte aligned
    if (T.rows_bytes % 128 || T.stage_bytes % 128) return false;
    T.nst = nst;
    T.rec_map = int(shapes.size());
    c->tm2 = T;
    c->tm2_box = shapes;
    return true;
}

// CTAs per SM of the two-nodes-per-thread kernel: one for tiles of 512
// nodes, two for tiles of 256 (each with half of the SM's tensor memory and
// shared memory)
int rows_pairs_ctas_per_sm(const sllbm_ctx* c) {
    int ty = 0, tz = 0;
    rows_pairs_shape(c->mesh.D, c->mesh.N[0], c->tm2.p, ty, tz);
    return c->mesh.N[0] * ty * tz == 256 ? 2 : 1;
}

// The pair structure the paired collision of the two-nodes-per-thread kernel
// assumes for D3Q45 (PairLayout<3>): base and opposite exactly negated, the
// pair's zero component exactly zero, equal weights within a shell, a rest
// velocity at index 0.
bool pair_layout_holds(const HostVelSet& vs) {
    using PL = PairLayout<3>;
    if (vs.Q != 2 * PL::NPAIR + 1 || vs.D != 3) return false;
    for (int d = 0; d < 3; ++d)
        if (vs.xi[d] != 0.0) return false;
    for (int k = 0; k < PL::NPAIR; ++k) {
        const int b = PL::base(k), o = PL::opp(b);
        for (int d = 0; d < 3; ++d) {
            if (vs.xi[o * 3 + d] != -vs.xi[b * 3 + d]) return false;
            if (PL::zero(b) == d && vs.xi[b * 3 + d] != 0.0) return false;
        }
        const int sh = VelSet<3>::shell(b);
        const int rep = PL::base(sh == 1 ? 0 : (sh == 2 ? 6 : 16));
        if (VelSet<3>::shell(o) != sh || vs.w[o] != vs.w[b] || vs.w[b] != vs.w[rep]) return false;
    }
    bool seen[64] = {};
    for (int i = 0; i < vs.Q; ++i) {
        const int sl = PL::slot(i);
        if (sl < 0 || sl >= vs.Q || seen[sl]) return false;
        seen[sl] = true;
    }
    return true;
}

// Tables of the row-tile kernel with two nodes per thread (step_tmem2.cuh):
// tiles of TY x TZ whole x rows.  Per (velocity, tile class): one box of
// source rows per population (the y range times the z range of the (y, z)
// taps of the tile's rows with non-zero weight: each row's taps are a product
// of y and z offsets, so the union is that box), copied by one TMA tensor
// copy; per tile row one record with the taps' slots and weights and the x
// weights of its even and odd nodes over six row sums; per tile class the
// velocities whose x factor is not the identity.  False where it does not apply.
bool build_rows_pairs(sllbm_ctx* c, const std::vector<TileRec<float>>& t, std::vector<int32_t>& head,
                      std::vector<TmRec2>& recs, std::vector<uint64_t>& xmask, std::vector<uint64_t>& smask) {
    const HostMesh& m = c->mesh;
    const StepGeom& G = c->geom;
    const int Q = c->vs.Q, D = m.D, NX = m.N[0], N1 = m.N[1], N2 = D == 3 ? m.N[2] : 1;
    int TY = 0, TZ = 0;
    if (c->precision != SLLBM_FP32 || m.p != 2 || !c->tiled || !c->row_uniform) return false;
    if (!((c->velset == SLLBM_D3Q45 && D == 3 && pair_layout_holds(c->vs)) || (c->velset == SLLBM_D2Q19 && D == 2)))
        return false;
    if (!rows_pairs_shape(D, NX, 2, TY, TZ) || G.ncls[0] != 2 || !m.periodic[0]) return false;
    const bool py = m.periodic[1] != 0;
    if (py && N1 % TY) return false;
    if (D == 3 && (!m.periodic[2] || N2 % TZ)) return false;
    if (int64_t(Q) * m.n_nodes >= (int64_t(1) << 31)) return false;
    const int NR = TY * TZ;
    TmGeom2 T{};
    T.ntile_y = (N1 + TY - 1) / TY;
    T.ntile_z = D == 3 ? N2 / TZ : 1;
    T.ntiles = T.ntile_y * T.ntile_z;
    // tile classes: node classes repeat with period 2 along a periodic axis,
    // so a tile's classes depend on its y tile (non-periodic y) or on the
    // parity of its first y, and on the parity of its first z
    T.ncy = py ? (TY % 2 ? 2 : 1) : T.ntile_y;
    T.ncz = D == 3 && TZ % 2 ? 2 : 1;
    T.n_tc = T.ncy * T.ncz;
    head.assign(size_t(Q) * T.n_tc * TM2_HEAD, 0);
    recs.assign(size_t(Q) * T.n_tc * NR, TmRec2{});
    xmask.assign(size_t(T.n_tc), 0);
    const int NRT = D == 3 ? 9 : 3;
    int max_rows = 1;
    std::vector<int> shapes;
    struct Tap {
        int src, dy, dz;
        float w;
    };
    struct Box {
        int src, ylo, yhi, zlo, zhi, slot;
    };
    for (int i = 0; i < Q; ++i)
        for (int tc = 0; tc < T.n_tc; ++tc) {
            const int y0 = (tc % T.ncy) * TY, z0 = (tc / T.ncy) * TZ;
            int32_t* h = &head[(size_t(i) * T.n_tc + tc) * TM2_HEAD];
            std::vector<std::vector<Tap>> taps(NR);
            std::vector<int> cls0(NR, -1);
            for (int r = 0; r < NR; ++r) {
                const int ry = r % TY, rz = r / TY;
                const int y = y0 + ry, z = z0 + rz;
                if (y >= N1) continue;                   // beyond a ragged last tile: an idle row
                cls0[r] = G.ncls[0] * ((py ? (y & 1) : y) + G.ncls[1] * (D == 3 ? (z & 1) : 0));
                const TileRec<float>& a = t[size_t(i) * G.n_classes + cls0[r]];
                if ((a.meta & 15) == REC_EQ) continue;
                for (int k = 0; k < NRT; ++k) {
                    const float wk = a.rw[k];
                    if (std::fabs(wk) < 1e-12f) continue;
                    const int dy = ((a.dyzp >> (4 * (k % 3))) & 15) - 8;
                    const int dz = D == 3 ? ((a.dyzp >> (12 + 4 * (k / 3))) & 15) - 8 : 0;
                    taps[r].push_back({a.meta >> 8, ry + dy, rz + dz, wk});
                }
            }
            std::vector<Box> boxes;
            for (int r = 0; r < NR; ++r)
                for (const Tap& tp : taps[r]) {
                    bool found = false;
                    for (Box& b : boxes)
                        if (b.src == tp.src) {
                            b.ylo = std::min(b.ylo, tp.dy);
                            b.yhi = std::max(b.yhi, tp.dy);
                            b.zlo = std::min(b.zlo, tp.dz);
                            b.zhi = std::max(b.zhi, tp.dz);
                            found = true;
                        }
                    if (!found) boxes.push_back({tp.src, tp.dy, tp.dy, tp.dz, tp.dz, 0});
                }
            if (int(boxes.size()) > TM2_MAX_BOXES) return false;
            int nrows = 0;
            for (size_t q = 0; q < boxes.size(); ++q) {
                Box& b = boxes[q];
                const int ny = b.yhi - b.ylo + 1, nz = b.zhi - b.zlo + 1;
                if (b.ylo + 128 < 0 || b.yhi + 128 > 255 || b.zlo + 128 < 0 || b.zhi + 128 > 255 || ny > 64 ||
                    nz > 64 || ny > N1 || nz > N2)
                    return false;
                int map = -1;
                for (size_t k = 0; k < shapes.size(); ++k)
                    if (shapes[k] == (ny | (nz << 8))) map = int(k);
                if (map < 0) {
                    if (int(shapes.size()) == TM2_MAX_MAPS - 1) return false;     // one map left for the records
                    map = int(shapes.size());
                    shapes.push_back(ny | (nz << 8));
                }
                b.slot = nrows;
                nrows += ny * nz;
                h[2 + q] = tm2_pack_box(b.src, b.ylo, b.zlo, map);
                h[2 + TM2_MAX_BOXES + q] = b.slot;
                h[2 + 2 * TM2_MAX_BOXES + q] = ny | (nz << 8);
            }
            if (nrows > TM2_MAX_ROWS) return false;
            h[0] = int(boxes.size());
            h[1] = nrows;
            max_rows = std::max(max_rows, nrows);
            bool xchg = false;
            for (int r = 0; r < NR; ++r) {
                TmRec2& ro = recs[(size_t(i) * T.n_tc + tc) * NR + r];
                ro.meta = REC_EQ;
                if (cls0[r] < 0) continue;              // an idle row
                const TileRec<float>& a = t[size_t(i) * G.n_classes + cls0[r]];
                ro.meta = a.meta;
                ro.ntap = int(taps[r].size());
                if ((a.meta & 15) == REC_EQ) continue;
                for (size_t q = 0; q < taps[r].size(); ++q) {
                    const Tap& tp = taps[r][q];
                    int sl = -1;
                    for (const Box& bx : boxes)
                        if (bx.src == tp.src) sl = bx.slot + (tp.dz - bx.zlo) * (bx.yhi - bx.ylo + 1) + (tp.dy - bx.ylo);
                    ro.off[q] = sl * NX * 8;
                    ro.w[q] = tp.w;
                }
                // x weights over the window of row sums: the even node x reads
                // x - 2 .. x + 2 (slots 0 .. 4), the odd node x + 1 reads
                // x - 1 .. x + 3 (its slots 0 .. 4); a tap at offset d from the
                // node sits in slot d + 2 of its window
                for (int xp = 0; xp < 2; ++xp) {
                    const TileRec<float>& b = t[size_t(i) * G.n_classes + cls0[r] + xp];
                    if (b.meta != a.meta) return false;
                    float* wx = xp ? ro.wxo : ro.wxe;
                    for (int q = 0; q < 3; ++q) {
                        const int d = ((b.dxp >> (4 * q)) & 15) - 8;
                        if (d < -2 || d > 2) return false;
                        wx[d + 2] += b.wx[q];
                    }
                    for (int q = 0; q < 5; ++q)
                        if (std::fabs(double(wx[q]) - (q == 2 ? 1.0 : 0.0)) > 1e-12) xchg = true;
                }
            }
            if (xchg) xmask[tc] |= uint64_t(1) << i;
        }
    T.p = 2;
    return pack_rows_pairs(c, T, NX, NR, max_rows, shapes, head, recs, smask);
}

// The same tables at order p = 4 from the order-P class records (TileRecP:
// factorised 1D weights, packed offsets).  Tiles of TY x TZ rows; on a
// periodic axis the classes of a tile's rows repeat with period 4 / gcd(4,
// extent), so tile classes are (y tile or y tile mod that period, z tile mod
// it).  Per row one 352-byte record: the (y, z) taps shared by all x classes
// (the class records guarantee it), and for each pair class (x mod 4 = 0, 2)
// the nine x weights of its even and odd node over ten row sums.
bool build_rows_pairs4(sllbm_ctx* c, const std::vector<TileRecP<float, 4>>& t, std::vector<int32_t>& head,
                       std::vector<TmRec4>& recs, std::vector<uint64_t>& xmask, std::vector<uint64_t>& smask) {
    const HostMesh& m = c->mesh;
    const StepGeom& G = c->geom;
    const int Q = c->vs.Q, D = m.D, NX = m.N[0], N1 = m.N[1], N2 = D == 3 ? m.N[2] : 1;
    constexpr int P = 4;
    int TY = 0, TZ = 0;
    if (c->precision != SLLBM_FP32 || m.p != P || D != 3 || c->velset != SLLBM_D3Q45 || !pair_layout_holds(c->vs))
        return false;
    if (!rows_pairs_shape(D, NX, P, TY, TZ) || G.ncls[0] != P || !m.periodic[0] || !m.periodic[2]) return false;
    const bool py = m.periodic[1] != 0;
    if ((py && N1 % TY) || N2 % TZ) return false;
    if (int64_t(Q) * m.n_nodes >= (int64_t(1) << 31)) return false;
    auto period = [](int extent) { return extent % 4 == 0 ? 1 : (extent % 2 == 0 ? 2 : 4); };
    const int NR = TY * TZ;
    TmGeom2 T{};
    T.ntile_y = (N1 + TY - 1) / TY;
    T.ntile_z = N2 / TZ;
    T.ntiles = T.ntile_y * T.ntile_z;
    T.ncy = py ? period(TY) : T.ntile_y;
    T.ncz = period(TZ);
    T.n_tc = T.ncy * T.ncz;
    T.p = P;
    const int64_t U = G.n_classes;
    head.assign(size_t(Q) * T.n_tc * TM2_HEAD, 0);
    recs.assign(size_t(Q) * T.n_tc * NR, TmRec4{});
    xmask.assign(size_t(T.n_tc), 0);
    int max_rows = 1;
    std::vector<int> shapes;
    struct Tap {
        int src, dy, dz;
        float w;
    };
    struct Box {
        int src, ylo, yhi, zlo, zhi, slot;
    };
    auto cls_of = [&](int kx, int y, int z) { return int64_t(kx) + G.ncls[0] * ((py ? y % P : y) + G.ncls[1] * (z % P)); };
    for (int i = 0; i < Q; ++i)
        for (int tc = 0; tc < T.n_tc; ++tc) {
            const int cy = tc % T.ncy, cz = tc / T.ncy;
            const int y0 = cy * TY, z0 = cz * TZ;       // a tile of this class
            int32_t* h = &head[(size_t(i) * T.n_tc + tc) * TM2_HEAD];
            std::vector<std::vector<Tap>> taps(NR);
            std::vector<int64_t> u0(NR, -1);
            for (int r = 0; r < NR; ++r) {
                const int ry = r % TY, rz = r / TY;
                const int y = y0 + ry, z = z0 + rz;
                if (y >= N1) continue;                   // beyond a ragged last tile: an idle row
                u0[r] = cls_of(0, y, z);
                const TileRecP<float, P>& a = t[size_t(i * U + u0[r])];
                if ((a.meta & 15) == REC_EQ) continue;
                for (int ka = 0; ka <= P; ++ka)
                    for (int kb = 0; kb <= P; ++kb) {
                        const float wk = a.wy[ka] * a.wz[kb];
                        if (std::fabs(wk) < 1e-12f) continue;
                        const int dy = ((a.dyp >> (4 * ka)) & 15) - 8;
                        const int dz = ((a.dzp >> (4 * kb)) & 15) - 8;
                        taps[r].push_back({a.meta >> 8, ry + dy, rz + dz, wk});
                    }
                if (taps[r].size() > 25) return false;
            }
            std::vector<Box> boxes;
            for (int r = 0; r < NR; ++r)
                for (const Tap& tp : taps[r]) {
                    bool found = false;
                    for (Box& b : boxes)
                        if (b.src == tp.src) {
                            b.ylo = std::min(b.ylo, tp.dy);
                            b.yhi = std::max(b.yhi, tp.dy);
                            b.zlo = std::min(b.zlo, tp.dz);
                            b.zhi = std::max(b.zhi, tp.dz);
                            found = true;
                        }
                    if (!found) boxes.push_back({tp.src, tp.dy, tp.dy, tp.dz, tp.dz, 0});
                }
            if (int(boxes.size()) > TM2_MAX_BOXES) return false;
            int nrows = 0;
            for (size_t q = 0; q < boxes.size(); ++q) {
                Box& b = boxes[q];
                const int ny = b.yhi - b.ylo + 1, nz = b.zhi - b.zlo + 1;
                if (b.ylo + 128 < 0 || b.yhi + 128 > 255 || b.zlo + 128 < 0 || b.zhi + 128 > 255 || ny > 64 ||
                    nz > 64 || ny > N1 || nz > N2)
                    return false;
                int map = -1;
                for (size_t k = 0; k < shapes.size(); ++k)
                    if (shapes[k] == (ny | (nz << 8))) map = int(k);
                if (map < 0) {
                    if (int(shapes.size()) == TM2_MAX_MAPS - 1) return false;     // one map left for the records
                    map = int(shapes.size());
                    shapes.push_back(ny | (nz << 8));
                }
                b.slot = nrows;
                nrows += ny * nz;
                h[2 + q] = tm2_pack_box(b.src, b.ylo, b.zlo, map);
                h[2 + TM2_MAX_BOXES + q] = b.slot;
                h[2 + 2 * TM2_MAX_BOXES + q] = ny | (nz << 8);
            }
            if (nrows > TM2_MAX_ROWS) return false;
            h[0] = int(boxes.size());
            h[1] = nrows;
            max_rows = std::max(max_rows, nrows);
            bool xchg = false;
            for (int r = 0; r < NR; ++r) {
                TmRec4& ro = recs[(size_t(i) * T.n_tc + tc) * NR + r];
                ro.meta = REC_EQ;
                if (u0[r] < 0) continue;                 // an idle row
                const TileRecP<float, P>& a = t[size_t(i * U + u0[r])];
                ro.meta = a.meta;
                ro.ntap = int(taps[r].size());
                if ((a.meta & 15) == REC_EQ) continue;
                for (size_t q = 0; q < taps[r].size(); ++q) {
                    const Tap& tp = taps[r][q];
                    int sl = -1;
                    for (const Box& bx : boxes)
                        if (bx.src == tp.src) sl = bx.slot + (tp.dz - bx.zlo) * (bx.yhi - bx.ylo + 1) + (tp.dy - bx.ylo);
                    ro.off[q] = sl * NX * 8;
                    ro.w[q] = tp.w;
                }
                // x weights: pair class pc (x mod 4 = 2 pc), node e (x + e):
                // a tap at offset d from node x + e sits in slot d + 4 of
                // that node's window (x - 4 + e .. x + 4 + e)
                const int ry = r % TY, rz = r / TY;
                for (int pc = 0; pc < 2; ++pc)
                    for (int e = 0; e < 2; ++e) {
                        const TileRecP<float, P>& b = t[size_t(i * U + cls_of(2 * pc + e, y0 + ry, z0 + rz))];
                        if (b.meta != a.meta) return false;
                        float* wx = ro.wx[pc][e];
                        for (int ka = 0; ka <= P; ++ka) {
                            const int d = ((b.dxp >> (4 * ka)) & 15) - 8;
                            if (d < -4 || d > 4) return false;
                            wx[d + 4] += b.wx[ka];
                        }
                        for (int q = 0; q < 9; ++q)
                            if (std::fabs(double(wx[q]) - (q == 4 ? 1.0 : 0.0)) > 1e-12) xchg = true;
                    }
            }
            if (xchg) xmask[tc] |= uint64_t(1) << i;
        }
    return pack_rows_pairs(c, T, NX, NR, max_rows, shapes, head, recs, smask);
}

// TMA tensor maps of the two-nodes-per-thread row-tile kernel: state buffer b
// viewed as the 4D FP32 tensor [Q][Nz][Ny][2 NX] (innermost last), one map
// per box shape {2 NX, rows along y, rows along z, 1}, then one of the
// records; maps[b * (shapes + 1) + k].
// The encoder comes from the driver through the runtime's entry-point query.
int encode_tm2_maps(sllbm_ctx* c) {
    const HostMesh& m = c->mesh;
    const int NX = m.N[0], N1 = m.N[1], N2 = m.D == 3 ? m.N[2] : 1, Q = c->vs.Q;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return fail(c, SLLBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const int nm = int(c->tm2_box.size());
    int ty = 0, tz = 0;
    rows_pairs_shape(m.D, NX, c->tm2.p, ty, tz);
    std::vector<CUtensorMap> maps(size_t(2) * (nm + 1));
    for (int b = 0; b < 2; ++b) {
        // the records [Q][n_tc][TY TZ] (128 or 352 bytes) as FP32
        // [Q][n_tc][TY TZ][32 or 88]: one box per (velocity, tile class)
        const int rf = c->tm2.p == 4 ? int(sizeof(TmRec4) / 4) : int(sizeof(TmRec2) / 4);   // floats per record
        const cuuint64_t rdims[4] = {cuuint64_t(rf), cuuint64_t(ty * tz), cuuint64_t(c->tm2.n_tc), cuuint64_t(Q)};
        const cuuint64_t rstrides[3] = {cuuint64_t(4 * rf), cuuint64_t(4 * rf) * ty * tz,
                                        cuuint64_t(4 * rf) * ty * tz * c->tm2.n_tc};
        const cuuint32_t rbox[4] = {cuuint32_t(rf), cuuint32_t(ty * tz), 1, 1};
        const cuuint32_t res[4] = {1, 1, 1, 1};
        const CUresult rr = enc(&maps[size_t(b) * (nm + 1) + nm], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->tm2_recs,
                                rdims, rstrides, rbox, res, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (rr != CUDA_SUCCESS)
            return fail(c, SLLBM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the records (code " +
                                               std::to_string(int(rr)) + ")");
        for (int k = 0; k < nm; ++k) {
            const cuuint64_t dims[4] = {cuuint64_t(2 * NX), cuuint64_t(N1), cuuint64_t(N2), cuuint64_t(Q)};
            const cuuint64_t strides[3] = {cuuint64_t(2 * NX) * 4, cuuint64_t(2 * NX) * N1 * 4,
                                           cuuint64_t(2 * NX) * N1 * N2 * 4};
            const cuuint32_t box[4] = {cuuint32_t(2 * NX), cuuint32_t(c->tm2_box[k] & 255),
                                       cuuint32_t(c->tm2_box[k] >> 8), 1};
            const cuuint32_t es[4] = {1, 1, 1, 1};
            const CUresult r = enc(&maps[size_t(b) * (nm + 1) + k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->fg[b],
                                   dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                return fail(c, SLLBM_ERR_CUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string(int(r)) + ")");
        }
    }
    cudaError_t e = dev_alloc(c, reinterpret_cast<void**>(&c->tm2_maps), sizeof(CUtensorMap) * maps.size());
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
    e = cudaMemcpyAsync(c->tm2_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                        c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy of the tensor maps");
    return SLLBM_OK;
}

template <typename real>
int dispatch_step(sllbm_ctx* ctx, const StepLaunch<real>& L) {
    const int vs = ctx->velset, p = ctx->mesh.p;
    if (ctx->generic) {
        ctx->step_kernel = "k_step_generic";
        return launch_step_generic<real>(p, ctx->mesh.D, L, static_cast<const GenVel<real>*>(ctx->gen_v), ctx->vs.Q);
    }
    const bool st = ctx->mode != SLLBM_STREAM_GATHER && ctx->mode != SLLBM_STREAM_GATHER_SMEM;
    if constexpr (std::is_same<real, float>::value) {
        if (st && ctx->rows_tm2 && !ctx->row_copy) {
            ctx->step_kernel = "k_step_rows_pairs";
            const int b = static_cast<const void*>(L.fg) == ctx->fg[0] ? 0 : 1;
            const char* maps = static_cast<const char*>(ctx->tm2_maps) +
                               size_t(b) * (ctx->tm2_box.size() + 1) * sizeof(CUtensorMap);
            return launch_rows_pairs(vs, ctx->mesh.N[0], L.fg, L.fgo, maps, ctx->tm2_head,
                                     ctx->tm2_recs, ctx->tm_xmask, ctx->tm2_smask, L.tw,
                                     L.G, *L.C, ctx->tm2, ctx->d_status, L.stream, ctx->tm_grid);
        }
        if (st && ctx->rows_tmem && !ctx->row_copy) {
            ctx->step_kernel = ctx->tm.kp ? "k_step_rows_tmem_tc" : "k_step_rows_tmem";
            return launch_rows_tmem(vs, ctx->mesh.N[0], L.fg, L.fgo, ctx->tm_bop, ctx->tm_head,
                                    static_cast<const TmRec*>(ctx->tm_recs), ctx->tm_xmask, L.tw, L.G, *L.C,
                                    ctx->tm, ctx->d_status, L.stream, ctx->tm_grid);
        }
        // a periodic row that fits one block exactly: one block per row, where
        // the block's shared memory still lets 16 warps reside per SM (D3Q45
        // rows of 192 nodes take 78 KB per block: 12 warps, slower than the
        // warp tiles)
        const int nx = ctx->mesh.N[0];
        if (st && ctx->tiled && ctx->row_copy && ctx->row_uniform && ctx->mode == SLLBM_STREAM_STRUCTURED &&
            (vs == 1 || vs == 3) && (nx == 32 || nx == 64 || nx == 128 || (nx == 256 && vs == 1))) {
            ctx->step_kernel = "k_step_row_copy";
            StepLaunch<real> Lc = L;
            Lc.status = ctx->d_status;
#define ROWCCASE(VS)                                                        \
    if (vs == VS) {                                                         \
        if (nx == 32) return launch_step_row_copy<VS, real, 32, 6>(Lc);     \
        if (nx == 64) return launch_step_row_copy<VS, real, 64, 6>(Lc);     \
        if (nx == 128) return launch_step_row_copy<VS, real, 128, 6>(Lc);   \
    }
            ROWCCASE(1)
            ROWCCASE(3)
#undef ROWCCASE
            return launch_step_row_copy<1, real, 256, 6>(Lc);
        }
        if (st && ctx->tiled && ctx->mode == SLLBM_STREAM_STRUCTURED && (vs == 1 || vs == 3) &&
            (nx == 32 || nx == 64 || nx == 128 || (nx == 192 && vs == 1) || nx == 256)) {
            ctx->step_kernel = "k_step_row_smem";
            StepLaunch<real> Lr = L;
            Lr.row = static_cast<const RowRec*>(ctx->row_tab);
#define ROWCASE(VS)                                                   \
    if (vs == VS) {                                                   \
        if (nx == 32) return launch_step_row_smem<VS, real, 32>(Lr);   \
        if (nx == 64) return launch_step_row_smem<VS, real, 64>(Lr);   \
        if (nx == 128) return launch_step_row_smem<VS, real, 128>(Lr); \
        if (nx == 192) return launch_step_row_smem<VS, real, 192>(Lr); \
        return launch_step_row_smem<VS, real, 256>(Lr);                \
    }
            ROWCASE(1)
            ROWCASE(3)
#undef ROWCASE
        }
    }
    if (st && ctx->tiled) {
        const bool reg = ctx->mode == SLLBM_STREAM_TILED_REG;
        ctx->step_kernel = reg ? "k_step_tiled" : "k_step_tiled_smem";
        switch (vs) {
            case 0: return reg ? launch_step_tiled<0, real>(L) : launch_step_tiled_smem<0, real>(L);
            case 1: return reg ? launch_step_tiled<1, real>(L) : launch_step_tiled_smem<1, real>(L);
            case 2: return reg ? launch_step_tiled<2, real>(L) : launch_step_tiled_smem<2, real>(L);
            case 3: return reg ? launch_step_tiled<3, real>(L) : launch_step_tiled_smem<3, real>(L);
        }
    }
    if (st && ctx->tiled_p == 4) {
        StepLaunch<real> Lp = L;
        Lp.tilep = ctx->tile_tab;
        if constexpr (std::is_same<real, float>::value) {
            // order 4, a periodic row that fits one block: one block per row
            const int nx = ctx->mesh.N[0];
            if ((vs == 1 || vs == 3) && (nx == 32 || nx == 64 || nx == 128 || nx == 256)) {
                ctx->step_kernel = "k_step_row_p";
#define ROWPCASE(VS)                                                     \
    if (vs == VS) {                                                      \
        if (nx == 32) return launch_step_row_p<VS, 4, real, 32>(Lp);     \
        if (nx == 64) return launch_step_row_p<VS, 4, real, 64>(Lp);     \
        if (nx == 128) return launch_step_row_p<VS, 4, real, 128>(Lp);   \
        return launch_step_row_p<VS, 4, real, 256>(Lp);                  \
    }
                ROWPCASE(1)
                ROWPCASE(3)
#undef ROWPCASE
            }
        }
        ctx->step_kernel = "k_step_tiled_p";
        switch (vs) {
            case 0: return launch_step_tiled_p<0, 4, real>(Lp);
            case 1: return launch_step_tiled_p<1, 4, real>(Lp);
            case 2: return launch_step_tiled_p<2, 4, real>(Lp);
            case 3: return launch_step_tiled_p<3, 4, real>(Lp);
        }
    }
    const bool gsm = ctx->mode == SLLBM_STREAM_GATHER_SMEM;
    ctx->step_kernel = st ? "k_step_structured" : (gsm ? "k_step_gather_smem" : "k_step_gather");
#define CASE(VS, P)                                                                                    \
    if (vs == VS && p == P)                                                                            \
        return st ? launch_step_structured<VS, P, real>(L)                                             \
                  : (gsm ? launch_step_gather_smem<VS, P, real>(L) : launch_step_gather<VS, P, real>(L));
    CASE(0, 2)
    CASE(1, 2)
    CASE(1, 3)
    CASE(2, 2)
    CASE(3, 2)
    CASE(0, 4)
    CASE(1, 4)
    CASE(2, 4)
#undef CASE
    if (vs == 3 && p == 4) {
        ctx->step_kernel = st ? "k_step_structured_smem" : "k_step_gather_smem";
        return st ? launch_step_structured_smem<3, 4, real>(L) : launch_step_gather_smem<3, 4, real>(L);
    }
    return fail(ctx, SLLBM_ERR_UNSUPPORTED,
                "velocity set / order combination not built (p must be 2 or 4, or 3 for D2Q19)");
}

bool supported(int vs, int p) {
    if (vs == SLLBM_D3Q125 || vs == SLLBM_VELSET_CUSTOM) return p >= 2 && p <= 4;     // the generic kernels
    return p == 2 || p == 4 || (vs == SLLBM_D2Q19 && p == 3);
}

// The warp-tiled kernel needs p = 2, periodic x, x-tap offsets within +-3
// nodes, and y/z factors (and record kinds) independent of the x parity.
bool tiled_eligible(const sllbm_ctx* c, const std::vector<Rec64>& rec) {
    const HostMesh& m = c->mesh;
    if (m.p != 2 || !m.periodic[0] || m.N[0] < 8) return false;
    if (int64_t(c->vs.Q) * m.n_nodes >= (int64_t(1) << 31)) return false;
    if (m.D == 3 && !m.periodic[2]) return false;
    const StepGeom& G = c->geom;
    const int64_t U = c->n_rec_units;
    for (int i = 0; i < c->vs.Q; ++i)
        for (int64_t u = 0; u < U; u += 2) {     // x parity is the fastest class index
            const Rec64& a = rec[size_t(i * U + u)];
            const Rec64& b = rec[size_t(i * U + u + 1)];
            if (a.meta != b.meta || (a.cell < 0) != (b.cell < 0)) return false;
            if (a.cell < 0) continue;
            const int64_t ya = (a.cell / m.cells[0]) % m.cells[1], yb = (b.cell / m.cells[0]) % m.cells[1];
            const int64_t za = a.cell / (int64_t(m.cells[0]) * m.cells[1]), zb = b.cell / (int64_t(m.cells[0]) * m.cells[1]);
            if (ya != yb || za != zb) return false;
            for (int d = 1; d < m.D; ++d)
                if (a.xi[d] != b.xi[d]) return false;
            for (int d = 1; d < m.D; ++d) {
                const int64_t cd = d == 1 ? ya : za;
                const int kd = int((u / (d == 1 ? G.ncls[0] : int64_t(G.ncls[0]) * G.ncls[1])) % G.ncls[d]);
                for (int t = 0; t <= 2; ++t) {
                    int64_t off = cd * 2 + t - kd;
                    if (m.periodic[d]) {                                         // nearest periodic image
                        if (off > m.N[d] / 2) off -= m.N[d];
                        if (off < -m.N[d] / 2) off += m.N[d];
                    }
                    if (m.periodic[d] && (off < -3 || off > 3)) return false;   // seam logic covers +-3
                    if (off < -7 || off > 7) return false;                       // 4-bit packing
                }
            }
            for (int par = 0; par < 2; ++par) {
                const Rec64& r = par ? b : a;
                const int cx = int(r.cell % m.cells[0]);
                for (int t = 0; t <= 2; ++t) {
                    int d = cx * 2 + t - par;
                    if (d > m.N[0] / 2) d -= m.N[0];
                    if (d < -m.N[0] / 2) d += m.N[0];
                    if (d < -3 || d > 3) return false;
                }
            }
        }
    (void)G;
    return true;
}

// The order-P warp-tiled kernel needs periodic x (and z in 3D), x taps within
// +-P lanes, (y, z) offsets within the 4-bit packing (+-7, and nearest image
// on periodic axes), and every x class of a (y, z) class sharing the record's
// kind, source, y / z cell and y / z reference coordinates.
template <int P>
bool tiled_p_eligible(const sllbm_ctx* c, const std::vector<Rec64>& rec) {
    const HostMesh& m = c->mesh;
    if (m.p != P || !m.periodic[0] || m.N[0] < 16) return false;
    if (int64_t(c->vs.Q) * m.n_nodes >= (int64_t(1) << 31)) return false;
    if (m.D == 3 && !m.periodic[2]) return false;
    const StepGeom& G = c->geom;
    if (G.ncls[0] != P) return false;
    const int64_t U = c->n_rec_units;
    const int64_t C01 = int64_t(m.cells[0]) * m.cells[1];
    for (int i = 0; i < c->vs.Q; ++i)
        for (int64_t u = 0; u < U; u += P) {     // x class is the fastest class index
            const Rec64& a = rec[size_t(i * U + u)];
            for (int k0 = 1; k0 < P; ++k0) {
                const Rec64& b = rec[size_t(i * U + u + k0)];
                if (a.meta != b.meta || (a.cell < 0) != (b.cell < 0)) return false;
                if (a.cell < 0) continue;
                if ((a.cell / m.cells[0]) % m.cells[1] != (b.cell / m.cells[0]) % m.cells[1] ||
                    a.cell / C01 != b.cell / C01)
                    return false;
                for (int d = 1; d < m.D; ++d)
                    if (a.xi[d] != b.xi[d]) return false;
            }
            if (a.cell < 0) continue;
            for (int d = 1; d < m.D; ++d) {
                const int64_t cd = d == 1 ? (a.cell / m.cells[0]) % m.cells[1] : a.cell / C01;
                const int kd = int((u / (d == 1 ? G.ncls[0] : int64_t(G.ncls[0]) * G.ncls[1])) % G.ncls[d]);
                for (int t = 0; t <= P; ++t) {
                    int64_t off = cd * P + t - kd;
                    if (m.periodic[d]) {
                        if (off > m.N[d] / 2) off -= m.N[d];
                        if (off < -m.N[d] / 2) off += m.N[d];
                        if (2 * (off < 0 ? -off : off) >= m.N[d]) return false;
                    }
                    if (off < -7 || off > 7) return false;
                }
            }
            for (int k0 = 0; k0 < P; ++k0) {
                const Rec64& r = rec[size_t(i * U + u + k0)];
                const int cx = int(r.cell % m.cells[0]);
                for (int t = 0; t <= P; ++t) {
                    int d = cx * P + t - k0;
                    if (d > m.N[0] / 2) d -= m.N[0];
                    if (d < -m.N[0] / 2) d += m.N[0];
                    if (d < -P || d > P) return false;
                }
            }
        }
    return true;
}

// Order-P warp-tiled records: x taps as lane offsets, (y, z) row offsets from
// the class's representative node (nearest image on periodic axes), and the
// factorised 1D Lagrange weights at the departure point's reference coordinates.
template <typename real, int P>
void build_tile_table_p(const sllbm_ctx* c, const std::vector<Rec64>& rec, std::vector<TileRecP<real, P>>& out) {
    const HostMesh& m = c->mesh;
    const StepGeom& G = c->geom;
    const int Q = c->vs.Q, D = m.D;
    const int64_t U = c->n_rec_units;
    out.assign(size_t(Q * U), TileRecP<real, P>());
    for (int i = 0; i < Q; ++i)
        for (int64_t u = 0; u < U; ++u) {
            const Rec64& r = rec[size_t(i * U + u)];
            TileRecP<real, P>& o = out[size_t(i * U + u)];
            std::memset(&o, 0, sizeof(o));
            o.meta = r.meta;
            if (r.cell < 0) continue;
            const int k[3] = {int(u % G.ncls[0]), int((u / G.ncls[0]) % G.ncls[1]),
                              int(u / (int64_t(G.ncls[0]) * G.ncls[1]))};
            const int cc[3] = {int(r.cell % m.cells[0]), int((r.cell / m.cells[0]) % m.cells[1]),
                               int(r.cell / (int64_t(m.cells[0]) * m.cells[1]))};
            int packed[3] = {0, 0, 0};
            for (int d = 0; d < D; ++d)
                for (int a = 0; a <= P; ++a) {
                    double v = 1.0;
                    for (int q = 0; q <= P; ++q)
                        if (q != a) v *= (r.xi[d] - m.glc[q]) / (m.glc[a] - m.glc[q]);
                    (d == 0 ? o.wx : d == 1 ? o.wy : o.wz)[a] = real(v);
                    int off = cc[d] * P + a - k[d];
                    if (m.periodic[d]) {
                        if (off > m.N[d] / 2) off -= m.N[d];
                        if (off < -m.N[d] / 2) off += m.N[d];
                    }
                    packed[d] |= (off + 8) << (4 * a);
                }
            o.dxp = packed[0];
            o.dyp = packed[1];
            o.dzp = packed[2];
        }
}

}  // namespace

// ====================================================================== API
extern "C" {

const char* sllbm_last_error(const sllbm_ctx* ctx) {
    return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

int sllbm_destroy(sllbm_ctx* ctx) {
    if (!ctx) return SLLBM_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->gen_v == ctx->gen_v64) ctx->gen_v = nullptr;       // one table in FP64 contexts
    void* ptrs[] = {ctx->dV[0], ctx->dV[1], ctx->dV[2], ctx->dX, ctx->rec64, ctx->cls_tab, ctx->g_code, ctx->g_xi,
                    ctx->tw_tab, ctx->fg[0], ctx->fg[1], ctx->tile_tab, ctx->row_tab, ctx->d_red, ctx->d_flag,
                    ctx->d_mom, ctx->mlp_img, ctx->d_feat, ctx->d_wref, ctx->mlp_tc, ctx->d_status,
                    ctx->d_plane, ctx->d_cp, ctx->d_plane_acc, ctx->tm_head, ctx->tm_recs, ctx->tm_xmask,
                    ctx->tm_bop, ctx->d_layers, ctx->tm2_head, ctx->tm2_recs, ctx->tm2_maps, ctx->tm2_smask,
                    ctx->gen_v, ctx->gen_v64};
    for (void* p : ptrs)
        if (p) dev_free(ctx, p);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return SLLBM_OK;
}

namespace {
// the allocator of contexts created from now on (sllbm_set_allocator)
sllbm_alloc_fn g_alloc_fn = nullptr;
sllbm_free_fn g_free_fn = nullptr;
void* g_alloc_user = nullptr;

// sllbm_create and sllbm_create_desc: `vs_in` is a checked caller's set
// (SLLBM_VELSET_CUSTOM), else the set of kind `velset` is built here
int create_ctx(const sllbm_mesh_desc* mesh, int32_t velset, const HostVelSet* vs_in, const sllbm_params* params,
               sllbm_ctx** out) {
    if (!out) return fail(nullptr, SLLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!mesh || !params) return fail(nullptr, SLLBM_ERR_ARG, "NULL descriptor");
    if (!(params->dt > 0) || !(params->gamma > 1.0) || !(params->Pr > 0) || !(params->mu_ref > 0) ||
        !(params->T_ref > 0))
        return fail(nullptr, SLLBM_ERR_ARG, "dt > 0, gamma > 1, Pr > 0, mu_ref > 0, T_ref > 0 required");
    if (params->precision != SLLBM_FP32 && params->precision != SLLBM_FP64)
        return fail(nullptr, SLLBM_ERR_ARG, "bad precision");

    sllbm_ctx* ctx = new (std::nothrow) sllbm_ctx();
    if (!ctx) return fail(nullptr, SLLBM_ERR_NOMEM, "host allocation failed");
    ctx->desc = *mesh;
    ctx->params = *params;
    ctx->velset = velset;
    ctx->device = params->device;
    ctx->precision = params->precision;
    auto bail = [&](int code) {
        g_create_error = ctx->last_error;
        sllbm_destroy(ctx);
        return code;
    };
    ctx->alloc_fn = g_alloc_fn;
    ctx->free_fn = g_free_fn;
    ctx->alloc_user = g_alloc_user;
    ctx->generic = velset == SLLBM_D3Q125 || velset == SLLBM_VELSET_CUSTOM;
    int rc = SLLBM_OK;
    if (vs_in)
        ctx->vs = *vs_in;
    else
        rc = build_velocity_set(velset, ctx->vs, ctx->last_error);
    if (rc) return bail(rc);
    rc = build_mesh(*mesh, ctx->mesh, ctx->last_error);
    if (rc) return bail(rc);
    if (ctx->vs.D != ctx->mesh.D) {
        ctx->last_error = "velocity set dimension differs from mesh dimension";
        return bail(SLLBM_ERR_ARG);
    }
    if (!supported(velset, ctx->mesh.p)) {
        ctx->last_error = ctx->generic ? "the generic velocity-set kernels are built for p = 2, 3, 4"
                                       : "velocity set / order combination not built (p must be 2, or 3 for D2Q19)";
        return bail(SLLBM_ERR_UNSUPPORTED);
    }
    for (int b = 0; b < 2; ++b) {
        const int k = mesh->bc[b].kind;
        if (k < 0 || k > SLLBM_BC_FARFIELD || !(mesh->bc[b].rho > 0) || !(mesh->bc[b].T > 0)) {
            ctx->last_error = "bad boundary descriptor";
            return bail(SLLBM_ERR_ARG);
        }
        if (ctx->mesh.kind != SLLBM_MESH_BOX && !(ctx->mesh.kind == SLLBM_MESH_EXPLICIT && ctx->mesh.periodic[1]) &&
            k == SLLBM_BC_PERIODIC) {
            ctx->last_error = "non-periodic boundary needs a boundary kind";
            return bail(SLLBM_ERR_ARG);
        }
    }
    // the host-side descriptors are checked; now the device
    {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            cudaGetLastError();
            ctx->last_error = "no CUDA device available";
            return bail(SLLBM_ERR_ARCH);
        }
        if (params->device < 0 || params->device >= ndev) {
            ctx->last_error = "bad device ordinal";
            return bail(SLLBM_ERR_ARG);
        }
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, params->device) != cudaSuccess) {
            ctx->last_error = "cudaGetDeviceProperties failed";
            return bail(SLLBM_ERR_CUDA);
        }
        if (!(prop.major == 10 && prop.minor == 3)) {
            ctx->last_error = "device is not compute capability 10.3 (sm_103)";
            return bail(SLLBM_ERR_ARCH);
        }
    }
    const bool axis = ctx->mesh.kind != SLLBM_MESH_NACA;
    int mode = params->stream_mode;
    if (mode == SLLBM_STREAM_AUTO) mode = axis ? SLLBM_STREAM_STRUCTURED : SLLBM_STREAM_GATHER;
    if (ctx->generic) mode = SLLBM_STREAM_GATHER;       // one departure record per (node, velocity)
    // the class records assume translation invariance along periodic
    // dimensions: a non-uniform one takes the gather streaming
    if (!ctx->mesh.uniform_periodic) mode = SLLBM_STREAM_GATHER;
    if (mode == SLLBM_STREAM_ROW_COPY) {
        ctx->row_copy = true;
        mode = SLLBM_STREAM_STRUCTURED;
    }
    // the row-tile kernels with the node state in tensor memory: requested
    // explicitly, or by default for the 45-velocity set on structured meshes
    // (faster there; the one-block-per-row kernel stays the default in 2D):
    // two nodes per thread where the rows allow it (64 or 128 nodes), else
    // one node per thread
    const bool d3_default = (mode == SLLBM_STREAM_AUTO || mode == SLLBM_STREAM_STRUCTURED) && velset == SLLBM_D3Q45;
    if (mode == SLLBM_STREAM_ROWS_TMEM || mode == SLLBM_STREAM_TENSOR || mode == SLLBM_STREAM_ROWS_PAIRS || d3_default)
        ctx->want_tmem = true;
    ctx->want_tc = mode == SLLBM_STREAM_TENSOR;
    ctx->want_tm2 = mode == SLLBM_STREAM_ROWS_PAIRS || d3_default;
    if (mode == SLLBM_STREAM_ROWS_TMEM || mode == SLLBM_STREAM_ROW_SMEM || mode == SLLBM_STREAM_TENSOR ||
        mode == SLLBM_STREAM_ROWS_PAIRS)
        mode = SLLBM_STREAM_STRUCTURED;
    if ((mode == SLLBM_STREAM_STRUCTURED || mode == SLLBM_STREAM_STRUCTURED_NODE || mode == SLLBM_STREAM_TILED_REG) &&
        !axis) {
        ctx->last_error = "structured streaming needs axis-aligned cells";
        return bail(SLLBM_ERR_ARG);
    }
    if (mode != SLLBM_STREAM_STRUCTURED && mode != SLLBM_STREAM_GATHER && mode != SLLBM_STREAM_STRUCTURED_NODE &&
        mode != SLLBM_STREAM_TILED_REG && mode != SLLBM_STREAM_GATHER_SMEM) {
        ctx->last_error = "bad stream mode";
        return bail(SLLBM_ERR_ARG);
    }
    ctx->mode = mode;
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        ctx->last_error = "cudaSetDevice failed";
        return bail(SLLBM_ERR_CUDA);
    }
    if (params->stream) {
        ctx->stream = static_cast<cudaStream_t>(params->stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            ctx->last_error = "cudaStreamCreate failed";
            return bail(SLLBM_ERR_CUDA);
        }
        ctx->own_stream = true;
    }
    fill_collide_const(ctx, ctx->cc32);
    fill_collide_const(ctx, ctx->cc64);
    rc = [&]() -> int {
        const HostMesh& m = ctx->mesh;
        const int Q = ctx->vs.Q, D = m.D;
        const int64_t N = m.n_nodes;
        cudaStream_t s = ctx->stream;
        // ---- geometry upload
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->dX), sizeof(double) * N * D));
        CK(cudaMemcpyAsync(ctx->dX, m.X.data(), sizeof(double) * N * D, cudaMemcpyHostToDevice, s));
        MeshView MV;
        std::memset(&MV, 0, sizeof(MV));
        MV.kind = m.kind;
        MV.D = D;
        MV.p = m.p;
        for (int d = 0; d < 3; ++d) {
            MV.cells[d] = m.cells[d];
            MV.N[d] = m.N[d];
            MV.periodic[d] = m.periodic[d];
            MV.length[d] = m.length[d];
        }
        if (axis)
            for (int d = 0; d < D; ++d) {
                CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->dV[d]), sizeof(double) * m.V[d].size()));
                CK(cudaMemcpyAsync(ctx->dV[d], m.V[d].data(), sizeof(double) * m.V[d].size(),
                                   cudaMemcpyHostToDevice, s));
                MV.V[d] = ctx->dV[d];
            }
        MV.X = ctx->dX;
        for (int a = 0; a <= m.p; ++a) {
            MV.glc[a] = m.glc[a];
            double den = 1.0;
            for (int q = 0; q <= m.p; ++q)
                if (q != a) den *= (m.glc[a] - m.glc[q]);
            MV.glc_inv_den[a] = 1.0 / den;
        }
        MV.bc_kind[0] = ctx->desc.bc[0].kind;
        MV.bc_kind[1] = ctx->desc.bc[1].kind;
        MV.R = m.length[1];
        TraceArgs A;
        std::memset(&A, 0, sizeof(A));
        A.M = MV;
        A.Q = Q;
        A.dt = params->dt;
        A.max_newton = params->max_newton > 0 ? params->max_newton : 40;
        A.max_walk = params->max_walk > 0 ? params->max_walk : 64;
        for (int i = 0; i < Q; ++i) {
            for (int d = 0; d < D; ++d) A.xi[i][d] = ctx->vs.xi[i * D + d];
            A.opp[i] = ctx->vs.opp[i];
        }
        // ---- geometry of the step kernels
        StepGeom& G = ctx->geom;
        std::memset(&G, 0, sizeof(G));
        G.n_nodes = N;
        G.n_classes = 1;
        for (int d = 0; d < 3; ++d) {
            G.N[d] = m.N[d];
            G.cells[d] = m.cells[d];
            G.periodic[d] = d < D ? m.periodic[d] : 0;
            G.ncls[d] = d < D ? (m.periodic[d] ? m.p : m.N[d]) : 1;
            G.n_classes *= G.ncls[d];
        }
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_status), 2 * sizeof(int)));       // status word, test wait limit
        CK(cudaMemsetAsync(ctx->d_status, 0, 2 * sizeof(int), ctx->stream));
#ifdef SLLBM_CHECKED
        G.status = ctx->d_status;
#endif
        const bool st = ctx->mode != SLLBM_STREAM_GATHER && ctx->mode != SLLBM_STREAM_GATHER_SMEM;
        ctx->n_rec_units = st ? G.n_classes : N;
        const int64_t U = ctx->n_rec_units;
        // ---- FP64 trace
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->rec64), sizeof(Rec64) * U * Q));
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_flag), sizeof(int) * 4));
        CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int) * 4, s));
        int r2 = launch_trace(A, ctx->dX, U, st ? 1 : 0, G.ncls[0], G.ncls[1], ctx->rec64, ctx->d_flag, s);
        if (r2) return fail(ctx, r2, "trace launch failed");
        int nfail = 0;
        CK(cudaMemcpyAsync(&nfail, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (nfail)
            return fail(ctx, SLLBM_ERR_DP_NOT_FOUND,
                        std::to_string(nfail) + " departure records not resolved within the Newton / walk caps");
        // ---- isothermal wall temperatures per unit
        double bcT[16];
        for (int k = 0; k < 16; ++k) bcT[k] = 1.0;
        bcT[0] = ctx->desc.bc[0].T;
        bcT[1] = ctx->desc.bc[1].T;
        double* d_bcT = nullptr;
        double* d_tw64 = nullptr;
        unsigned long long* d_cnt = nullptr;
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&d_bcT), sizeof(bcT)));
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&d_tw64), sizeof(double) * U));
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&d_cnt), sizeof(unsigned long long) * 2));
        CK(cudaMemcpyAsync(d_bcT, bcT, sizeof(bcT), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * 2, s));
        r2 = launch_isothermal(ctx->rec64, U, Q, d_bcT, d_tw64, d_cnt, s);
        if (r2) return fail(ctx, r2, "isothermal launch failed");
        std::vector<double> tw(U);
        unsigned long long cnt[2];
        CK(cudaMemcpyAsync(tw.data(), d_tw64, sizeof(double) * U, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        dev_free(ctx, d_bcT);
        dev_free(ctx, d_tw64);
        dev_free(ctx, d_cnt);
        ctx->n_boundary_records = int64_t(cnt[0]);
        ctx->n_isothermal_nodes = int64_t(cnt[1]);
        if (st) {   // isothermal count per node = per class x class multiplicity
            int64_t mult = 1;
            for (int d = 0; d < D; ++d)
                if (m.periodic[d]) mult *= m.N[d] / m.p;
            ctx->n_boundary_records *= mult;
            ctx->n_isothermal_nodes *= mult;
        }
        const size_t rs = real_size(ctx);
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tw_tab), rs * U));
        if (rs == 8) {
            CK(cudaMemcpyAsync(ctx->tw_tab, tw.data(), 8 * U, cudaMemcpyHostToDevice, s));
        } else {
            std::vector<float> tw32(U);
            for (int64_t u = 0; u < U; ++u) tw32[u] = float(tw[u]);
            CK(cudaMemcpyAsync(ctx->tw_tab, tw32.data(), 4 * U, cudaMemcpyHostToDevice, s));
            CK(cudaStreamSynchronize(s));
        }
        // ---- step tables
        if (st) {
            std::vector<Rec64> rec(size_t(U * Q));
            CK(cudaMemcpyAsync(rec.data(), ctx->rec64, sizeof(Rec64) * U * Q, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            ctx->tiled = (ctx->mode == SLLBM_STREAM_STRUCTURED || ctx->mode == SLLBM_STREAM_TILED_REG) &&
                         tiled_eligible(ctx, rec);
            if ((ctx->mode == SLLBM_STREAM_STRUCTURED || ctx->mode == SLLBM_STREAM_TILED_REG) &&
                ctx->mesh.p == 4 && tiled_p_eligible<4>(ctx, rec)) {
                if (rs == 8) {
                    std::vector<TileRecP<double, 4>> t;
                    build_tile_table_p(ctx, rec, t);
                    CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tile_tab), sizeof(t[0]) * t.size()));
                    CK(cudaMemcpyAsync(ctx->tile_tab, t.data(), sizeof(t[0]) * t.size(), cudaMemcpyHostToDevice, s));
                } else {
                    std::vector<TileRecP<float, 4>> t;
                    build_tile_table_p(ctx, rec, t);
                    CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tile_tab), sizeof(t[0]) * t.size()));
                    CK(cudaMemcpyAsync(ctx->tile_tab, t.data(), sizeof(t[0]) * t.size(), cudaMemcpyHostToDevice, s));
                    // the two-nodes-per-thread row tiles at order 4
                    std::vector<int32_t> th;
                    std::vector<TmRec4> tr4;
                    std::vector<uint64_t> tx, ts;
                    if (ctx->want_tm2 && build_rows_pairs4(ctx, t, th, tr4, tx, ts)) {
                        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm2_smask), sizeof(uint64_t) * ts.size()));
                        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm2_head), sizeof(int32_t) * th.size()));
                        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm2_recs), sizeof(TmRec4) * tr4.size()));
                        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm_xmask), sizeof(uint64_t) * tx.size()));
                        CK(cudaMemcpyAsync(ctx->tm2_smask, ts.data(), sizeof(uint64_t) * ts.size(),
                                           cudaMemcpyHostToDevice, s));
                        CK(cudaMemcpyAsync(ctx->tm2_head, th.data(), sizeof(int32_t) * th.size(),
                                           cudaMemcpyHostToDevice, s));
                        CK(cudaMemcpyAsync(ctx->tm2_recs, tr4.data(), sizeof(TmRec4) * tr4.size(),
                                           cudaMemcpyHostToDevice, s));
                        CK(cudaMemcpyAsync(ctx->tm_xmask, tx.data(), sizeof(uint64_t) * tx.size(),
                                           cudaMemcpyHostToDevice, s));
                        CK(cudaStreamSynchronize(s));
                        int sms = 0;
                        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
                        ctx->tm_grid = std::min(ctx->tm2.ntiles, sms * rows_pairs_ctas_per_sm(ctx));
                        ctx->rows_tm2 = true;
                    }
                }
                CK(cudaStreamSynchronize(s));
                ctx->tiled_p = 4;
            }
            if (ctx->tiled) {
                if (rs == 8) {
                    std::vector<TileRec<double>> t;
                    build_tile_table(ctx, rec, t);
                    CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tile_tab), sizeof(TileRec<double>) * t.size()));
                    CK(cudaMemcpyAsync(ctx->tile_tab, t.data(), sizeof(TileRec<double>) * t.size(),
                                       cudaMemcpyHostToDevice, s));
                } else {
                    std::vector<TileRec<float>> t;
                    build_tile_table(ctx, rec, t);
                    ctx->row_uniform = row_uniform_table(ctx, t);
                    std::vector<RowRec> rr(t.size());
                    for (size_t k = 0; k < t.size(); ++k) {
                        RowRec& o = rr[k];
                        o.meta = t[k].meta;
                        o.dxp = t[k].dxp;
                        o.dyzp = t[k].dyzp;
                        for (int q = 0; q < 9; ++q) {
                            o.rel[q] = t[k].rel[q];
                            o.rw[q] = t[k].rw[q];
                        }
                        for (int q = 0; q < 3; ++q) o.wx[q] = t[k].wx[q];
                    }
                    CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->row_tab), sizeof(RowRec) * rr.size()));
                    CK(cudaMemcpyAsync(ctx->row_tab, rr.data(), sizeof(RowRec) * rr.size(), cudaMemcpyHostToDevice, s));
                    CK(cudaStreamSynchronize(s));
                    std::vector<int32_t> th;
                    std::vector<TmRec> tr;
                    std::vector<uint64_t> tx;
                    std::vector<float> tb;
                    std::vector<TmRec2> tr2;
                    std::vector<uint64_t> ts;
                    if (ctx->want_tm2 && build_rows_pairs(ctx, t, th, tr2, tx, ts)) {
                        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm2_smask), sizeof(uint64_t) * ts.size()));
                        CK(cudaMemcpyAsync(ctx->tm2_smask, ts.data(), sizeof(uint64_t) * ts.size(),
                                           cudaMemcpyHostToDevice, s));
                        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm2_head), sizeof(int32_t) * th.size()));
                        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm2_recs), sizeof(TmRec2) * tr2.size()));
                        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm_xmask), sizeof(uint64_t) * tx.size()));
                        CK(cudaMemcpyAsync(ctx->tm2_head, th.data(), sizeof(int32_t) * th.size(),
                                           cudaMemcpyHostToDevice, s));
                        CK(cudaMemcpyAsync(ctx->tm2_recs, tr2.data(), sizeof(TmRec2) * tr2.size(),
                                           cudaMemcpyHostToDevice, s));
                        CK(cudaMemcpyAsync(ctx->tm_xmask, tx.data(), sizeof(uint64_t) * tx.size(),
                                           cudaMemcpyHostToDevice, s));
                        CK(cudaStreamSynchronize(s));
                        int sms = 0;
                        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
                        ctx->tm_grid = std::min(ctx->tm2.ntiles, sms * rows_pairs_ctas_per_sm(ctx));
                        ctx->rows_tm2 = true;
                        th.clear();
                        tx.clear();
                    }
                    if (!ctx->rows_tm2 && ctx->want_tmem && build_rows_tmem(ctx, t, th, tr, tx, tb)) {
                        if (!tb.empty()) {
                            CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm_bop), sizeof(float) * tb.size()));
                            CK(cudaMemcpyAsync(ctx->tm_bop, tb.data(), sizeof(float) * tb.size(),
                                               cudaMemcpyHostToDevice, s));
                        }
                        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm_head), sizeof(int32_t) * th.size()));
                        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm_recs), sizeof(TmRec) * tr.size()));
                        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tm_xmask), sizeof(uint64_t) * tx.size()));
                        CK(cudaMemcpyAsync(ctx->tm_head, th.data(), sizeof(int32_t) * th.size(),
                                           cudaMemcpyHostToDevice, s));
                        CK(cudaMemcpyAsync(ctx->tm_recs, tr.data(), sizeof(TmRec) * tr.size(),
                                           cudaMemcpyHostToDevice, s));
                        CK(cudaMemcpyAsync(ctx->tm_xmask, tx.data(), sizeof(uint64_t) * tx.size(),
                                           cudaMemcpyHostToDevice, s));
                        CK(cudaStreamSynchronize(s));
                        int sms = 0;
                        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
                        ctx->tm_grid = std::min(ctx->tm.ntiles, sms);
                        ctx->rows_tmem = true;
                    }
                    CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->tile_tab), sizeof(TileRec<float>) * t.size()));
                    CK(cudaMemcpyAsync(ctx->tile_tab, t.data(), sizeof(TileRec<float>) * t.size(),
                                       cudaMemcpyHostToDevice, s));
                }
                CK(cudaStreamSynchronize(s));
            }
            if (rs == 8) {
                std::vector<ClassRec<double>> t;
                build_class_table(ctx, rec, t);
                CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->cls_tab), sizeof(ClassRec<double>) * t.size()));
                CK(cudaMemcpyAsync(ctx->cls_tab, t.data(), sizeof(ClassRec<double>) * t.size(),
                                   cudaMemcpyHostToDevice, s));
                ctx->table_bytes = int64_t(sizeof(ClassRec<double>) * t.size());
                CK(cudaStreamSynchronize(s));
            } else {
                std::vector<ClassRec<float>> t;
                build_class_table(ctx, rec, t);
                CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->cls_tab), sizeof(ClassRec<float>) * t.size()));
                CK(cudaMemcpyAsync(ctx->cls_tab, t.data(), sizeof(ClassRec<float>) * t.size(),
                                   cudaMemcpyHostToDevice, s));
                ctx->table_bytes = int64_t(sizeof(ClassRec<float>) * t.size());
                CK(cudaStreamSynchronize(s));
            }
        } else {
            CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->g_code), sizeof(int32_t) * N * Q));
            CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->g_xi), rs * N * Q * D));
            ctx->table_bytes = int64_t((4 + rs * D) * N * Q);
            r2 = rs == 8 ? launch_pack_gather<double>(ctx->rec64, N, Q, D, ctx->g_code, (double*)ctx->g_xi, s)
                         : launch_pack_gather<float>(ctx->rec64, N, Q, D, ctx->g_code, (float*)ctx->g_xi, s);
            if (r2) return fail(ctx, r2, "pack launch failed");
        }
        // ---- state buffers
        for (int b = 0; b < 2; ++b) {
            CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->fg[b]), 2 * rs * N * Q));
        }
        if (ctx->generic) {
            // the generic kernels' per-velocity table, in the context's
            // precision and in FP64 (initialisation, moments, conservation)
            std::vector<GenVel<double>> g64;
            build_gen_table<double>(ctx, g64);
            CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->gen_v64), sizeof(GenVel<double>) * g64.size()));
            CK(cudaMemcpyAsync(ctx->gen_v64, g64.data(), sizeof(GenVel<double>) * g64.size(), cudaMemcpyHostToDevice,
                               s));
            if (rs == 8) {
                ctx->gen_v = ctx->gen_v64;
            } else {
                std::vector<GenVel<float>> g32;
                build_gen_table<float>(ctx, g32);
                CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->gen_v), sizeof(GenVel<float>) * g32.size()));
                CK(cudaMemcpyAsync(ctx->gen_v, g32.data(), sizeof(GenVel<float>) * g32.size(),
                                   cudaMemcpyHostToDevice, s));
            }
        }
        if (ctx->rows_tm2) {
            const int r3 = encode_tm2_maps(ctx);          // the maps name the state buffers
            if (r3 != SLLBM_OK) return r3;
        }
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_red), sizeof(double) * (conserve_blocks() * 5 + 8)));
        CK(cudaStreamSynchronize(s));
        return SLLBM_OK;
    }();
    if (rc) return bail(rc);
    *out = ctx;
    return SLLBM_OK;
}
}  // namespace

int sllbm_set_allocator(sllbm_alloc_fn alloc, sllbm_free_fn release, void* user) {
    if ((alloc == nullptr) != (release == nullptr))
        return fail(nullptr, SLLBM_ERR_ARG, "sllbm_set_allocator needs both functions, or neither");
    g_alloc_fn = alloc;
    g_free_fn = release;
    g_alloc_user = alloc ? user : nullptr;
    return SLLBM_OK;
}

int sllbm_create(const sllbm_mesh_desc* mesh, int32_t velset, const sllbm_params* params, sllbm_ctx** out) {
    if (velset == SLLBM_VELSET_CUSTOM) {
        if (out) *out = nullptr;
        return fail(nullptr, SLLBM_ERR_ARG, "a custom velocity set needs sllbm_create_desc");
    }
    return create_ctx(mesh, velset, nullptr, params, out);
}

int sllbm_create_desc(const sllbm_mesh_desc* mesh, const sllbm_velset_desc* velset, const sllbm_params* params,
                      sllbm_ctx** out) {
    if (out) *out = nullptr;
    if (!velset) return fail(nullptr, SLLBM_ERR_ARG, "NULL velocity-set descriptor");
    if (velset->kind != SLLBM_VELSET_CUSTOM) return create_ctx(mesh, velset->kind, nullptr, params, out);
    // a caller's set is copied and checked before any device work
    HostVelSet vs;
    std::string err;
    const int rc = build_custom_velocity_set(*velset, vs, err);
    if (rc) return fail(nullptr, rc, err);
    return create_ctx(mesh, SLLBM_VELSET_CUSTOM, &vs, params, out);
}

int sllbm_info(const sllbm_ctx* ctx, sllbm_info_t* o) {
    if (!ctx || !o) return SLLBM_ERR_ARG;
    std::memset(o, 0, sizeof(*o));
    o->n_nodes = ctx->mesh.n_nodes;
    o->Q = ctx->vs.Q;
    o->dim = ctx->mesh.D;
    o->p = ctx->mesh.p;
    for (int d = 0; d < 3; ++d) {
        o->nodes[d] = ctx->mesh.N[d];
        o->cells[d] = ctx->mesh.cells[d];
    }
    o->precision = ctx->precision;
    o->stream_mode = ((ctx->mode == SLLBM_STREAM_STRUCTURED || ctx->mode == SLLBM_STREAM_TILED_REG) && !ctx->tiled &&
                      !ctx->tiled_p)
                         ? SLLBM_STREAM_STRUCTURED_NODE
                         : (ctx->row_copy ? SLLBM_STREAM_ROW_COPY
                                          : (ctx->rows_tm2 ? SLLBM_STREAM_ROWS_PAIRS
                                             : (ctx->rows_tmem ? (ctx->tm.kp ? SLLBM_STREAM_TENSOR
                                                                             : SLLBM_STREAM_ROWS_TMEM)
                                                               : ctx->mode)));
    o->state_bytes = int64_t(2 * real_size(ctx) * ctx->mesh.n_nodes * ctx->vs.Q);
    o->table_bytes = ctx->table_bytes;
    o->n_records = int64_t(ctx->mesh.n_nodes) * ctx->vs.Q;
    o->n_boundary_records = ctx->n_boundary_records;
    o->n_isothermal_nodes = ctx->n_isothermal_nodes;
    std::strncpy(o->step_kernel, ctx->step_kernel, sizeof(o->step_kernel) - 1);
    o->step_kernel[sizeof(o->step_kernel) - 1] = 0;
    return SLLBM_OK;
}

int sllbm_node_coords(sllbm_ctx* ctx, double* x, int32_t on_device) {
    if (!ctx || !x) return SLLBM_ERR_ARG;
    cudaSetDevice(ctx->device);
    const size_t bytes = sizeof(double) * ctx->mesh.n_nodes * ctx->mesh.D;
    CK(cudaMemcpyAsync(x, ctx->dX, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SLLBM_OK;
}

int sllbm_velocity_set(const sllbm_ctx* ctx, double* xi, double* w, int32_t* opp) {
    if (!ctx) return SLLBM_ERR_ARG;
    const int Q = ctx->vs.Q, D = ctx->vs.D;
    if (xi) std::memcpy(xi, ctx->vs.xi.data(), sizeof(double) * Q * D);
    if (w) std::memcpy(w, ctx->vs.w.data(), sizeof(double) * Q);
    if (opp)
        for (int i = 0; i < Q; ++i) opp[i] = ctx->vs.opp[i];
    return SLLBM_OK;
}

int sllbm_init_state(sllbm_ctx* ctx, const double* rho, const double* u, const double* T, int32_t on_device) {
    if (!ctx || !rho || !u || !T) return SLLBM_ERR_ARG;
    cudaSetDevice(ctx->device);
    const int64_t N = ctx->mesh.n_nodes;
    const int D = ctx->mesh.D;
    cudaStream_t s = ctx->stream;
    const double *dr = rho, *du = u, *dT = T;
    double* tmp = nullptr;
    if (!on_device) {
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&tmp), sizeof(double) * N * (D + 2)));
        CK(cudaMemcpyAsync(tmp, rho, sizeof(double) * N, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(tmp + N, u, sizeof(double) * N * D, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(tmp + N * (D + 1), T, sizeof(double) * N, cudaMemcpyHostToDevice, s));
        dr = tmp;
        du = tmp + N;
        dT = tmp + N * (D + 1);
    }
    const GenVel<double>* gv = static_cast<const GenVel<double>*>(ctx->gen_v64);
    const int Qg = ctx->vs.Q, Dg = ctx->mesh.D;
    int rc = ctx->generic
                 ? (ctx->precision == SLLBM_FP64
                        ? launch_init_generic<double>(dr, du, dT, N, gv, Qg, Dg, (double2*)ctx->fg[0], s)
                        : launch_init_generic<float>(dr, du, dT, N, gv, Qg, Dg, (float2*)ctx->fg[0], s))
             : ctx->precision == SLLBM_FP64
                 ? launch_init<double>(ctx->velset, dr, du, dT, N, ctx->cc64, (double2*)ctx->fg[0], s)
                 : launch_init<float>(ctx->velset, dr, du, dT, N, ctx->cc64, (float2*)ctx->fg[0], s);
    if (tmp) {
        CK(cudaStreamSynchronize(s));
        dev_free(ctx, tmp);
    }
    if (rc) return fail(ctx, rc, "init launch failed");
    ctx->cur = 0;
    ctx->steps = 0;
    ctx->initialised = true;
    return SLLBM_OK;
}

namespace {
int state_io(sllbm_ctx* ctx, double* f, double* g, const double* cf, const double* cg, int32_t on_device, int dir) {
    cudaSetDevice(ctx->device);
    const int64_t N = ctx->mesh.n_nodes;
    const int Q = ctx->vs.Q;
    cudaStream_t s = ctx->stream;
    const size_t bytes = sizeof(double) * N * Q;
    double* buf = nullptr;
    CK(dev_alloc(ctx, reinterpret_cast<void**>(&buf), 2 * bytes + sizeof(double) * 2 * Q));
    double* dw = buf + 2 * N * Q;
    std::vector<double> wv(2 * Q);
    const double gf = 2.0 / (ctx->params.gamma - 1.0) - ctx->mesh.D;
    for (int i = 0; i < Q; ++i) {
        wv[i] = ctx->vs.w[i];
        wv[Q + i] = ctx->vs.w[i] * gf;
    }
    CK(cudaMemcpyAsync(dw, wv.data(), sizeof(double) * 2 * Q, cudaMemcpyHostToDevice, s));
    const cudaMemcpyKind k_in = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind k_out = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (dir == 1) {
        CK(cudaMemcpyAsync(buf, cf, bytes, k_in, s));
        CK(cudaMemcpyAsync(buf + N * Q, cg, bytes, k_in, s));
    }
    const int c = ctx->cur;
    int rc = ctx->precision == SLLBM_FP64
                 ? launch_convert<double>((double2*)ctx->fg[c], buf, buf + N * Q, N, Q, dw, dw + Q, dir, s)
                 : launch_convert<float>((float2*)ctx->fg[c], buf, buf + N * Q, N, Q, dw, dw + Q, dir, s);
    if (rc == SLLBM_OK && dir == 0) {
        if (f) CK(cudaMemcpyAsync(f, buf, bytes, k_out, s));
        if (g) CK(cudaMemcpyAsync(g, buf + N * Q, bytes, k_out, s));
    }
    CK(cudaStreamSynchronize(s));
    dev_free(ctx, buf);
    return rc ? fail(ctx, rc, "convert launch failed") : SLLBM_OK;
}
}  // namespace

int sllbm_get_state(sllbm_ctx* ctx, double* f, double* g, int32_t on_device) {
    if (!ctx) return SLLBM_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, SLLBM_ERR_STATE, "state not initialised");
    return state_io(ctx, f, g, nullptr, nullptr, on_device, 0);
}

int sllbm_set_state(sllbm_ctx* ctx, const double* f, const double* g, int32_t on_device) {
    if (!ctx || !f || !g) return SLLBM_ERR_ARG;
    ctx->cur = 0;
    int rc = state_io(ctx, nullptr, nullptr, f, g, on_device, 1);
    if (rc) return rc;
    ctx->steps = 0;
    ctx->initialised = true;
    return SLLBM_OK;
}

int sllbm_get_state_raw(sllbm_ctx* ctx, void* fg, int32_t on_device) {
    if (!ctx || !fg) return SLLBM_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, SLLBM_ERR_STATE, "state not initialised");
    cudaSetDevice(ctx->device);
    const size_t bytes = 2 * real_size(ctx) * ctx->mesh.n_nodes * ctx->vs.Q;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(fg, ctx->fg[ctx->cur], bytes, k, ctx->stream));
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
    return SLLBM_OK;
}

int sllbm_set_state_raw(sllbm_ctx* ctx, const void* fg, int32_t on_device) {
    if (!ctx || !fg) return SLLBM_ERR_ARG;
    cudaSetDevice(ctx->device);
    const size_t bytes = 2 * real_size(ctx) * ctx->mesh.n_nodes * ctx->vs.Q;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    ctx->cur = 0;
    CK(cudaMemcpyAsync(ctx->fg[0], fg, bytes, k, ctx->stream));
    ctx->steps = 0;
    ctx->initialised = true;
    return SLLBM_OK;
}

namespace {
// one launch of the fused step; mlpm: 0 plain (or learned if enabled), 2 export features
int step_once(sllbm_ctx* ctx, float* feat) {
    const int a = ctx->cur, b = 1 - a;
    const int mlpm = feat ? 2 : (ctx->mlp_enabled ? 1 : 0);
    int rc;
    if (ctx->precision == SLLBM_FP64) {
        if (mlpm) return fail(ctx, SLLBM_ERR_UNSUPPORTED, "learned collision runs in FP32");
        StepLaunch<double> L{(const double2*)ctx->fg[a], (double2*)ctx->fg[b], (const ClassRec<double>*)ctx->cls_tab,
                             (const TileRec<double>*)ctx->tile_tab, ctx->g_code, (const double*)ctx->g_xi,
                             (const double*)ctx->tw_tab, nullptr, nullptr, ctx->geom, &ctx->cc64, ctx->stream};
        rc = dispatch_step<double>(ctx, L);
    } else {
        StepLaunch<float> L{(const float2*)ctx->fg[a], (float2*)ctx->fg[b], (const ClassRec<float>*)ctx->cls_tab,
                            (const TileRec<float>*)ctx->tile_tab, ctx->g_code, (const float*)ctx->g_xi,
                            (const float*)ctx->tw_tab, ctx->mlp_img, feat, ctx->geom, &ctx->cc32, ctx->stream};
        if (mlpm) {
            if (!(ctx->tiled && ctx->velset == SLLBM_D2Q19))
                return fail(ctx, SLLBM_ERR_UNSUPPORTED,
                            "learned collision is built for D2Q19 with the warp-tiled structured kernel");
            ctx->step_kernel = mlpm == 1 && ctx->mlp_tensor ? "k_step_tiled_smem_tc" : "k_step_tiled";
            if (mlpm == 2) {
                rc = launch_step_tiled<1, float, 2>(L);
            } else if (ctx->mlp_tensor) {
                L.mlp_tc = ctx->mlp_tc;
                L.status = ctx->d_status;
                rc = launch_step_tiled_smem_tc<1, float>(L);
            } else {
                rc = launch_step_tiled<1, float, 1>(L);
            }
        } else {
            rc = dispatch_step<float>(ctx, L);
        }
    }
    if (rc) return rc == SLLBM_ERR_CUDA ? fail(ctx, rc, "step launch failed") : rc;
    ctx->cur = b;
    ++ctx->steps;
    return SLLBM_OK;
}
}  // namespace

int sllbm_step(sllbm_ctx* ctx, int64_t n) {
    if (!ctx || n < 0) return SLLBM_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, SLLBM_ERR_STATE, "state not initialised");
    cudaSetDevice(ctx->device);
    for (int64_t k = 0; k < n; ++k) {
        const int rc = step_once(ctx, nullptr);
        if (rc) return rc;
    }
    return SLLBM_OK;
}

int sllbm_step_features(sllbm_ctx* ctx, float* z, int32_t on_device) {
    if (!ctx || !z) return SLLBM_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, SLLBM_ERR_STATE, "state not initialised");
    cudaSetDevice(ctx->device);
    int rc = ensure_mlp_image(ctx);
    if (rc) return rc;
    const size_t bytes = sizeof(float) * ctx->mesh.n_nodes * ctx->vs.Q;
    float* dz = z;
    if (!on_device) {
        if (!ctx->d_feat) CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_feat), bytes));
        dz = ctx->d_feat;
    }
    rc = step_once(ctx, dz);
    if (rc) return rc;
    if (!on_device) {
        CK(cudaMemcpyAsync(z, dz, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return SLLBM_OK;
}

int sllbm_mlp_set(sllbm_ctx* ctx, const uint16_t* w_bf16, const float* biases, const float* s_in, float sigma,
                  int32_t enable) {
    if (!ctx) return SLLBM_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (!enable) {
        ctx->mlp_enabled = false;
        return SLLBM_OK;
    }
    if (!w_bf16 || !biases || !s_in || !(sigma > 0)) return SLLBM_ERR_ARG;
    if (ctx->precision != SLLBM_FP32 || !(ctx->tiled && ctx->velset == SLLBM_D2Q19))
        return fail(ctx, SLLBM_ERR_UNSUPPORTED,
                    "learned collision is built for FP32 D2Q19 contexts with the warp-tiled structured kernel");
    int rc = ensure_mlp_image(ctx);
    if (rc) return rc;
    const int Q = ctx->vs.Q, H = MLP_H;
    std::vector<float> img(ctx->mlp_host);
    auto f32 = [](uint16_t b) {
        const uint32_t u = uint32_t(b) << 16;
        float f;
        std::memcpy(&f, &u, 4);
        return f;
    };
    int k = 0;
    for (int p = 0; p < H * Q + H * H + Q * H; ++p) img[k++] = f32(w_bf16[p]);
    for (int p = 0; p < 2 * H + Q; ++p) img[k++] = biases[p];
    for (int q = 0; q < Q; ++q) img[k++] = s_in[q];
    img[img.size() - 1] = sigma;
    // the same weights as BF16 operand tiles of the tensor-core path:
    // W1 [64][K1], W2 [64][64], W3 [N3][64], zero padded, canonical K-major
    using TC = MlpTc<19, 2>;
    std::vector<uint16_t> tiles(TC::B_BYTES / 2, 0);
    auto put = [&](int base_bytes, int r, int kk, int K, uint16_t v) {
        tiles[(base_bytes + tc_canon_offset(r, kk, K)) / 2] = v;
    };
    const uint16_t* W1 = w_bf16;
    const uint16_t* W2 = W1 + H * Q;
    const uint16_t* W3 = W2 + H * H;
    for (int j = 0; j < H; ++j)
        for (int q = 0; q < Q; ++q) put(0, j, q, TC::K1, W1[j * Q + q]);
    for (int j = 0; j < H; ++j)
        for (int q = 0; q < H; ++q) put(TC::B1, j, q, H, W2[j * H + q]);
    for (int i = 0; i < Q; ++i)
        for (int q = 0; q < H; ++q) put(TC::B1 + TC::B2, i, q, H, W3[i * H + q]);
    if (!ctx->mlp_tc) CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->mlp_tc), TC::B_BYTES));
    if (!ctx->d_status) {
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_status), 2 * sizeof(int)));
        CK(cudaMemsetAsync(ctx->d_status, 0, 2 * sizeof(int), ctx->stream));
    }
    CK(cudaMemcpyAsync(ctx->mlp_tc, tiles.data(), TC::B_BYTES, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->mlp_img, img.data(), sizeof(float) * img.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->mlp_enabled = true;
    return SLLBM_OK;
}

int sllbm_mlp_path(sllbm_ctx* ctx, int32_t path) {
    if (!ctx || (path != SLLBM_MLP_TENSOR && path != SLLBM_MLP_SIMT)) return SLLBM_ERR_ARG;
    ctx->mlp_tensor = path == SLLBM_MLP_TENSOR;
    return SLLBM_OK;
}

int sllbm_device_status(sllbm_ctx* ctx, int32_t* code) {
    if (!ctx || !code) return SLLBM_ERR_ARG;
    *code = 0;
    cudaSetDevice(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    if (!ctx->d_status) return SLLBM_OK;
    int v = 0;
    CK(cudaMemcpy(&v, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(ctx->d_status, 0, sizeof(int)));
    *code = v;
    return SLLBM_OK;
}

int sllbm_debug_wait_limit(sllbm_ctx* ctx, int32_t log2_cycles) {
    if (!ctx || log2_cycles < 0 || log2_cycles > 31) return SLLBM_ERR_ARG;
    if (!ctx->d_status) return fail(ctx, SLLBM_ERR_STATE, "context has no status words");
    cudaSetDevice(ctx->device);
    CK(cudaMemcpyAsync(ctx->d_status + 1, &log2_cycles, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SLLBM_OK;
}

int sllbm_build_flags(void) {
#ifdef SLLBM_CHECKED
    return SLLBM_BUILD_CHECKED;
#else
    return 0;
#endif
}

int sllbm_moment_basis(const sllbm_ctx* ctx, double* Phi, double* P) {
    if (!ctx) return SLLBM_ERR_ARG;
    std::vector<double> ph, gi, pp;
    build_moment_basis(ctx->vs, ph, gi, pp);
    if (Phi) std::memcpy(Phi, ph.data(), sizeof(double) * ph.size());
    if (P) std::memcpy(P, pp.data(), sizeof(double) * pp.size());
    return SLLBM_OK;
}

int sllbm_step_count(const sllbm_ctx* ctx, int64_t* out) {
    if (!ctx || !out) return SLLBM_ERR_ARG;
    *out = ctx->steps;
    return SLLBM_OK;
}

int sllbm_read_moments(sllbm_ctx* ctx, double* rho, double* u, double* T, int32_t on_device) {
    if (!ctx) return SLLBM_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, SLLBM_ERR_STATE, "state not initialised");
    cudaSetDevice(ctx->device);
    const int64_t N = ctx->mesh.n_nodes;
    const int D = ctx->mesh.D;
    cudaStream_t s = ctx->stream;
    double *dr = rho, *du = u, *dT = T, *tmp = nullptr;
    if (!on_device) {
        if (!ctx->d_mom) CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_mom), sizeof(double) * N * (D + 2)));
        tmp = ctx->d_mom;
        dr = rho ? tmp : nullptr;
        du = u ? tmp + N : nullptr;
        dT = T ? tmp + N * (D + 1) : nullptr;
    }
    const int c = ctx->cur;
    const GenVel<double>* gv = static_cast<const GenVel<double>*>(ctx->gen_v64);
    int rc = ctx->generic
                 ? (ctx->precision == SLLBM_FP64
                        ? launch_moments_generic<double>((double2*)ctx->fg[c], N, gv, ctx->vs.Q, D, ctx->cc64.cv, dr,
                                                         du, dT, s)
                        : launch_moments_generic<float>((float2*)ctx->fg[c], N, gv, ctx->vs.Q, D, ctx->cc64.cv, dr, du,
                                                        dT, s))
             : ctx->precision == SLLBM_FP64
                 ? launch_moments<double>(ctx->velset, (double2*)ctx->fg[c], N, ctx->cc64, dr, du, dT, s)
                 : launch_moments_f32(ctx->velset, (float2*)ctx->fg[c], N, ctx->cc32, ctx->cc64.cv, dr, du, dT, s);
    if (rc) return fail(ctx, rc, "moments launch failed");
    if (!on_device) {
        if (rho) CK(cudaMemcpyAsync(rho, dr, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
        if (u) CK(cudaMemcpyAsync(u, du, sizeof(double) * N * D, cudaMemcpyDeviceToHost, s));
        if (T) CK(cudaMemcpyAsync(T, dT, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return SLLBM_OK;
}

int sllbm_conservation(sllbm_ctx* ctx, double* out) {
    if (!ctx || !out) return SLLBM_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, SLLBM_ERR_STATE, "state not initialised");
    cudaSetDevice(ctx->device);
    const int64_t N = ctx->mesh.n_nodes;
    const int D = ctx->mesh.D;
    cudaStream_t s = ctx->stream;
    double* part = ctx->d_red;
    double* dout = ctx->d_red + conserve_blocks() * 5;
    CK(cudaMemsetAsync(ctx->d_flag + 1, 0, sizeof(int), s));
    const int c = ctx->cur;
    int rc;
    if (ctx->generic) {
        const GenVel<double>* gv = static_cast<const GenVel<double>*>(ctx->gen_v64);
        const unsigned nb = unsigned(conserve_blocks());
        rc = ctx->precision == SLLBM_FP64
                 ? launch_conserve_generic<double>((double2*)ctx->fg[c], N, gv, ctx->vs.Q, D, ctx->cc64.cv, 1, nb,
                                                   part, ctx->d_flag + 1, s)
                 : launch_conserve_generic<float>((float2*)ctx->fg[c], N, gv, ctx->vs.Q, D, ctx->cc64.cv, 1, nb,
                                                  part, ctx->d_flag + 1, s);
        if (!rc) {
            k_reduce_parts_launch(part, int(nb), D + 2, dout, s);
            rc = cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
        }
    } else {
        rc = ctx->precision == SLLBM_FP64
                 ? launch_conserve<double>(ctx->velset, D, (double2*)ctx->fg[c], N, ctx->cc64, part,
                                           ctx->d_flag + 1, dout, s)
                 : launch_conserve<float>(ctx->velset, D, (float2*)ctx->fg[c], N, ctx->cc64, part,
                                          ctx->d_flag + 1, dout, s);
    }
    if (rc) return fail(ctx, rc, "conservation launch failed");
    int flag = 0;
    CK(cudaMemcpyAsync(out, dout, sizeof(double) * (D + 2), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&flag, ctx->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (flag) return fail(ctx, SLLBM_ERR_UNSTABLE, "non-positive density or temperature, or non-finite state");
    return SLLBM_OK;
}

int sllbm_departure_records(sllbm_ctx* ctx, int32_t* kind, int32_t* src, int32_t* bid, int32_t* cell, double* xi,
                            double* xsrc) {
    if (!ctx) return SLLBM_ERR_ARG;
    cudaSetDevice(ctx->device);
    const HostMesh& m = ctx->mesh;
    const int Q = ctx->vs.Q, D = m.D;
    const int64_t N = m.n_nodes, U = ctx->n_rec_units;
    std::vector<Rec64> rec(size_t(U * Q));
    CK(cudaMemcpyAsync(rec.data(), ctx->rec64, sizeof(Rec64) * U * Q, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const bool st = ctx->mode != SLLBM_STREAM_GATHER && ctx->mode != SLLBM_STREAM_GATHER_SMEM;
    for (int i = 0; i < Q; ++i)
        for (int64_t n = 0; n < N; ++n) {
            int k[3] = {0, 0, 0};
            int64_t r = n;
            for (int d = 0; d < D; ++d) {
                k[d] = int(r % m.N[d]);
                r /= m.N[d];
            }
            int64_t u = n;
            if (st) {
                const StepGeom& G = ctx->geom;
                int cl[3] = {0, 0, 0};
                for (int d = 0; d < D; ++d) cl[d] = m.periodic[d] ? k[d] % m.p : k[d];
                u = cl[0] + int64_t(G.ncls[0]) * (cl[1] + int64_t(G.ncls[1]) * cl[2]);
            }
            const Rec64& R = rec[size_t(i * U + u)];
            const int64_t o = i * N + n;
            const int kd = R.meta & 15;
            const int b = (R.meta >> 4) & 15;
            if (kind) kind[o] = kd;
            if (src) src[o] = (R.meta >> 8) & 255;
            if (bid) bid[o] = b == 15 ? -1 : b;
            int cc[3] = {0, 0, 0};
            if (R.cell >= 0) {
                int64_t cl = R.cell;
                for (int d = 0; d < D; ++d) {
                    cc[d] = int(cl % m.cells[d]);
                    cl /= m.cells[d];
                }
                if (st)
                    for (int d = 0; d < D; ++d)
                        if (m.periodic[d]) {
                            const int home = k[d] / m.p;
                            cc[d] = ((cc[d] + home) % m.cells[d] + m.cells[d]) % m.cells[d];
                        }
            }
            int64_t lin = -1;
            if (R.cell >= 0) lin = cc[0] + int64_t(m.cells[0]) * (cc[1] + int64_t(m.cells[1]) * cc[2]);
            if (cell) cell[o] = int32_t(lin);
            for (int d = 0; d < D; ++d) {
                if (xi) xi[o * D + d] = R.xi[d];
                if (xsrc) {
                    if (!st || R.cell < 0) {
                        xsrc[o * D + d] = R.xsrc[d];
                    } else {
                        const auto& V = m.V[d];
                        xsrc[o * D + d] = V[cc[d]] + 0.5 * (R.xi[d] + 1.0) * (V[cc[d] + 1] - V[cc[d]]);
                    }
                }
            }
        }
    return SLLBM_OK;
}

namespace {
// pack (dir 0) or unpack (dir 1) node layers x0 .. x0 + nx - 1 of the current state
int x_layers(sllbm_ctx* ctx, int32_t x0, int32_t nx, void* buf, int32_t on_device, int dir) {
    if (!ctx || !buf || nx <= 0 || x0 < 0 || x0 + nx > ctx->mesh.N[0]) return SLLBM_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, SLLBM_ERR_STATE, "state not initialised");
    cudaSetDevice(ctx->device);
    const HostMesh& m = ctx->mesh;
    const int rows = m.N[1] * (m.D == 3 ? m.N[2] : 1);
    const size_t bytes = 2 * real_size(ctx) * size_t(ctx->vs.Q) * rows * nx;
    void* dbuf = buf;
    if (!on_device) {
        if (ctx->layer_bytes < bytes) {
            if (ctx->d_layers) dev_free(ctx, ctx->d_layers);
            ctx->d_layers = nullptr;
            ctx->layer_bytes = 0;
            CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_layers), bytes));
            ctx->layer_bytes = bytes;
        }
        dbuf = ctx->d_layers;
        if (dir == 1) CK(cudaMemcpyAsync(dbuf, buf, bytes, cudaMemcpyHostToDevice, ctx->stream));
    }
    const int rc = ctx->precision == SLLBM_FP64
                       ? launch_x_layers<double2>((double2*)ctx->fg[ctx->cur], (double2*)dbuf, m.n_nodes, m.N[0],
                                                  rows, x0, nx, ctx->vs.Q, dir, ctx->stream)
                       : launch_x_layers<float2>((float2*)ctx->fg[ctx->cur], (float2*)dbuf, m.n_nodes, m.N[0], rows,
                                                 x0, nx, ctx->vs.Q, dir, ctx->stream);
    if (rc) return fail(ctx, rc, "layer copy launch failed");
    if (!on_device) {
        if (dir == 0) CK(cudaMemcpyAsync(buf, dbuf, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return SLLBM_OK;
}
}  // namespace

int sllbm_get_x_layers(sllbm_ctx* ctx, int32_t x0, int32_t nx, void* buf, int32_t on_device) {
    return x_layers(ctx, x0, nx, buf, on_device, 0);
}

int sllbm_set_x_layers(sllbm_ctx* ctx, int32_t x0, int32_t nx, const void* buf, int32_t on_device) {
    return x_layers(ctx, x0, nx, const_cast<void*>(buf), on_device, 1);
}

int sllbm_sync(sllbm_ctx* ctx) {
    if (!ctx) return SLLBM_ERR_ARG;
    cudaSetDevice(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    return SLLBM_OK;
}

void* sllbm_stream(const sllbm_ctx* ctx) { return ctx ? static_cast<void*>(ctx->stream) : nullptr; }

}  // extern "C"

// ====================================================================== forcing, mass rescaling, control
extern "C" {

int sllbm_set_force(sllbm_ctx* ctx, const double* F) {
    if (!ctx || !F) return SLLBM_ERR_ARG;
    for (int d = 0; d < 3; ++d) {
        if (!std::isfinite(F[d])) return fail(ctx, SLLBM_ERR_ARG, "force must be finite");
        ctx->force[d] = d < ctx->mesh.D ? F[d] : 0.0;
    }
    fill_collide_const(ctx, ctx->cc32);
    fill_collide_const(ctx, ctx->cc64);
    return SLLBM_OK;
}

int sllbm_rescale_mass(sllbm_ctx* ctx, double target_mass) {
    if (!ctx || !(target_mass > 0)) return SLLBM_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, SLLBM_ERR_STATE, "state not initialised");
    double sums[5];
    int rc = sllbm_conservation(ctx, sums);
    if (rc) return rc;
    const double s = target_mass / sums[0];
    cudaSetDevice(ctx->device);
    const int64_t N = ctx->mesh.n_nodes;
    const int Q = ctx->vs.Q;
    if (!ctx->d_wref) {
        std::vector<double> wv(2 * Q);
        const double gf = 2.0 / (ctx->params.gamma - 1.0) - ctx->mesh.D;
        for (int i = 0; i < Q; ++i) {
            wv[i] = ctx->vs.w[i];
            wv[Q + i] = ctx->vs.w[i] * gf;
        }
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_wref), sizeof(double) * 2 * Q));
        CK(cudaMemcpy(ctx->d_wref, wv.data(), sizeof(double) * 2 * Q, cudaMemcpyHostToDevice));
    }
    const int c = ctx->cur;
    rc = ctx->precision == SLLBM_FP64
             ? launch_scale_state<double>((double2*)ctx->fg[c], N, Q, ctx->d_wref, ctx->d_wref + Q, s, ctx->stream)
             : launch_scale_state<float>((float2*)ctx->fg[c], N, Q, ctx->d_wref, ctx->d_wref + Q, s, ctx->stream);
    return rc ? fail(ctx, rc, "rescale launch failed") : SLLBM_OK;
}

int sllbm_step_controlled(sllbm_ctx* ctx, int64_t n, const sllbm_control* cfg, double* force_out) {
    if (!ctx || !cfg || n < 0) return SLLBM_ERR_ARG;
    if (cfg->control_every < 0 || cfg->rescale_every < 0) return SLLBM_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, SLLBM_ERR_STATE, "state not initialised");
    const int D = ctx->mesh.D;
    const double Nn = double(ctx->mesh.n_nodes);
    for (int64_t k = 0; k < n; ++k) {
        int rc = sllbm_step(ctx, 1);
        if (rc) return rc;
        const int64_t s = ctx->steps;
        if (cfg->control_every > 0 && s % cfg->control_every == 0) {
            double sums[5];
            rc = sllbm_conservation(ctx, sums);
            if (rc) return rc;
            // PI control of the mean streamwise momentum density (nodal mean of rho u_x)
            const double err = cfg->target_momentum - sums[1] / Nn;
            ctx->ctl_integral += err * cfg->control_every * ctx->params.dt;
            double F[3] = {ctx->force[0], ctx->force[1], D == 3 ? ctx->force[2] : 0.0};
            F[0] = cfg->force0 + cfg->kp * err + cfg->ki * ctx->ctl_integral;
            rc = sllbm_set_force(ctx, F);
            if (rc) return rc;
        }
        if (cfg->rescale_every > 0 && s % cfg->rescale_every == 0) {
            rc = sllbm_rescale_mass(ctx, cfg->target_mass);
            if (rc) return rc;
        }
    }
    if (force_out)
        for (int d = 0; d < 3; ++d) force_out[d] = ctx->force[d];
    return SLLBM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ flow statistics (Sec. 4.2-4.4)
namespace {
// moments of the current state into ctx->d_mom: rho [N] | u [N][D] | T [N]
int moments_on_device(sllbm_ctx* ctx, double*& r, double*& u, double*& T) {
    const int64_t N = ctx->mesh.n_nodes;
    const int D = ctx->mesh.D;
    if (!ctx->d_mom) CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_mom), sizeof(double) * N * (D + 2)));
    r = ctx->d_mom;
    u = ctx->d_mom + N;
    T = ctx->d_mom + N * (D + 1);
    return sllbm_read_moments(ctx, r, u, T, 1);
}

int plane_checks(sllbm_ctx* ctx) {
    if (!ctx->initialised) return fail(ctx, SLLBM_ERR_STATE, "state not initialised");
    if (ctx->mesh.kind == SLLBM_MESH_NACA)
        return fail(ctx, SLLBM_ERR_UNSUPPORTED, "plane statistics need an axis-aligned mesh (box, channel, mixing)");
    return SLLBM_OK;
}

// plane means S [N1][K] (see stats.cu for the order of the K values)
int plane_means(sllbm_ctx* ctx, std::vector<double>& S) {
    int rc = plane_checks(ctx);
    if (rc) return rc;
    cudaSetDevice(ctx->device);
    const HostMesh& m = ctx->mesh;
    const int K = plane_stat_count(m.D);
    double *r = nullptr, *u = nullptr, *T = nullptr;
    rc = moments_on_device(ctx, r, u, T);
    if (rc) return rc;
    if (!ctx->d_plane) CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_plane), sizeof(double) * m.N[1] * K));
    rc = launch_plane_sums(r, u, T, m.D, m.N[0], m.N[1], m.D == 3 ? m.N[2] : 1, ctx->d_plane, 0, ctx->stream);
    if (rc) return fail(ctx, rc, "plane statistics launch failed");
    S.assign(size_t(m.N[1]) * K, 0.0);
    CK(cudaMemcpyAsync(S.data(), ctx->d_plane, sizeof(double) * S.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SLLBM_OK;
}

// increasing-power coefficients of the Lagrange polynomial a on the nodes xh
std::vector<double> lagrange_coeffs(const std::vector<double>& xh, int a) {
    std::vector<double> c(1, 1.0);
    for (int q = 0; q < int(xh.size()); ++q) {
        if (q == a) continue;
        const double s = 1.0 / (xh[a] - xh[q]);
        std::vector<double> nc(c.size() + 1, 0.0);
        for (size_t k = 0; k < c.size(); ++k) {
            nc[k + 1] += c[k] * s;
            nc[k] -= c[k] * xh[q] * s;
        }
        c.swap(nc);
    }
    return c;
}
}  // namespace

namespace {
// profiles from plane means S [N1][K] (instantaneous or averaged over time)
void derive_profiles(const sllbm_ctx* ctx, const std::vector<double>& S, double* y, double* rho_bar, double* u_bar,
                     double* u_favre, double* T_bar, double* p_bar, double* R) {
    const HostMesh& m = ctx->mesh;
    const int D = m.D, K = plane_stat_count(D);
    for (int j = 0; j < m.N[1]; ++j) {
        const double* s = &S[size_t(j) * K];
        const double rb = s[0];
        double uf[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) uf[a] = s[1 + a] / rb;
        if (y) y[j] = m.X[size_t(m.N[0]) * j * D + 1];
        if (rho_bar) rho_bar[j] = rb;
        for (int a = 0; a < D; ++a) {
            if (u_bar) u_bar[j * D + a] = s[1 + D + a];
            if (u_favre) u_favre[j * D + a] = uf[a];
        }
        if (T_bar) T_bar[j] = s[1 + 2 * D];
        if (p_bar) p_bar[j] = s[2 + 2 * D];
        if (R) {
            int k = 3 + 2 * D;
            for (int a = 0; a < D; ++a)
                for (int b = a; b < D; ++b, ++k) {
                    const double v = s[k] / rb - uf[a] * uf[b];
                    R[(size_t(j) * D + a) * D + b] = v;
                    R[(size_t(j) * D + b) * D + a] = v;
                }
        }
    }
}
}  // namespace

int sllbm_plane_profiles(sllbm_ctx* ctx, double* y, double* rho_bar, double* u_bar, double* u_favre, double* T_bar,
                         double* p_bar, double* R) {
    if (!ctx) return SLLBM_ERR_ARG;
    std::vector<double> S;
    int rc = plane_means(ctx, S);
    if (rc) return rc;
    derive_profiles(ctx, S, y, rho_bar, u_bar, u_favre, T_bar, p_bar, R);
    return SLLBM_OK;
}

int sllbm_stats_accumulate(sllbm_ctx* ctx) {
    if (!ctx) return SLLBM_ERR_ARG;
    int rc = plane_checks(ctx);
    if (rc) return rc;
    cudaSetDevice(ctx->device);
    const HostMesh& m = ctx->mesh;
    const int K = plane_stat_count(m.D);
    if (!ctx->d_plane_acc) {
        CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_plane_acc), sizeof(double) * m.N[1] * K));
        CK(cudaMemsetAsync(ctx->d_plane_acc, 0, sizeof(double) * m.N[1] * K, ctx->stream));
        ctx->stats_samples = 0;
    }
    double *r = nullptr, *u = nullptr, *T = nullptr;
    rc = moments_on_device(ctx, r, u, T);
    if (rc) return rc;
    rc = launch_plane_sums(r, u, T, m.D, m.N[0], m.N[1], m.D == 3 ? m.N[2] : 1, ctx->d_plane_acc, 1, ctx->stream);
    if (rc) return fail(ctx, rc, "plane statistics launch failed");
    ++ctx->stats_samples;
    return SLLBM_OK;
}

int sllbm_stats_reset(sllbm_ctx* ctx) {
    if (!ctx) return SLLBM_ERR_ARG;
    ctx->stats_samples = 0;
    if (ctx->d_plane_acc) {
        cudaSetDevice(ctx->device);
        CK(cudaMemsetAsync(ctx->d_plane_acc, 0, sizeof(double) * ctx->mesh.N[1] * plane_stat_count(ctx->mesh.D),
                           ctx->stream));
    }
    return SLLBM_OK;
}

int sllbm_plane_profiles_mean(sllbm_ctx* ctx, double* y, double* rho_bar, double* u_bar, double* u_favre,
                              double* T_bar, double* p_bar, double* R, int64_t* samples) {
    if (!ctx) return SLLBM_ERR_ARG;
    if (samples) *samples = ctx->stats_samples;
    if (ctx->stats_samples == 0) return fail(ctx, SLLBM_ERR_STATE, "no state accumulated (sllbm_stats_accumulate)");
    cudaSetDevice(ctx->device);
    const HostMesh& m = ctx->mesh;
    const int K = plane_stat_count(m.D);
    std::vector<double> S(size_t(m.N[1]) * K);
    CK(cudaMemcpyAsync(S.data(), ctx->d_plane_acc, sizeof(double) * S.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (double& v : S) v /= double(ctx->stats_samples);
    derive_profiles(ctx, S, y, rho_bar, u_bar, u_favre, T_bar, p_bar, R);
    return SLLBM_OK;
}

int sllbm_mixing_thickness(sllbm_ctx* ctx, double du, double rho0, double* delta_theta, double* delta_omega) {
    if (!ctx || !(du != 0.0) || !(rho0 > 0.0) || (!delta_theta && !delta_omega)) return SLLBM_ERR_ARG;
    std::vector<double> S;
    int rc = plane_means(ctx, S);
    if (rc) return rc;
    const HostMesh& m = ctx->mesh;
    const int D = m.D, K = plane_stat_count(D), p = m.p, N1 = m.N[1];
    // integral over [-1, 1] of each basis polynomial, and their derivatives at the nodes
    std::vector<double> Wint(p + 1, 0.0), dL((p + 1) * (p + 1), 0.0);
    for (int a = 0; a <= p; ++a) {
        const std::vector<double> c = lagrange_coeffs(m.glc, a);
        for (int k = 0; k < int(c.size()); k += 2) Wint[a] += 2.0 * c[k] / (k + 1);
        for (int q = 0; q <= p; ++q) {
            double v = 0.0, xp = 1.0;
            for (int k = 1; k < int(c.size()); ++k, xp *= m.glc[q]) v += k * c[k] * xp;
            dL[q * (p + 1) + a] = v;
        }
    }
    double theta = 0.0, slope = 0.0;
    for (int c = 0; c < m.cells[1]; ++c) {
        const double h = m.V[1][c + 1] - m.V[1][c];
        for (int q = 0; q <= p; ++q) {
            const int j = (c * p + q) % N1;
            const double* s = &S[size_t(j) * K];
            const double uf = s[1] / s[0];
            theta += 0.5 * h * Wint[q] * s[0] * (0.5 * du - uf) * (0.5 * du + uf);
            double d = 0.0;
            for (int b = 0; b <= p; ++b) d += dL[q * (p + 1) + b] * S[size_t((c * p + b) % N1) * K + 1 + D];
            slope = std::max(slope, std::fabs(d) * 2.0 / h);
        }
    }
    if (delta_theta) *delta_theta = theta / (rho0 * du * du);
    if (delta_omega) *delta_omega = slope > 0.0 ? du / slope : std::numeric_limits<double>::infinity();
    return SLLBM_OK;
}

int sllbm_plane_cp(sllbm_ctx* ctx, int32_t side, double p0, double mach, double* x, double* cp, int64_t* count) {
    if (!ctx || (side != 0 && side != 1) || !(p0 > 0.0) || !(mach > 0.0)) return SLLBM_ERR_ARG;
    const HostMesh& m = ctx->mesh;
    const int N2 = m.D == 3 ? m.N[2] : 1;
    const int64_t M = int64_t(m.N[0]) * N2;
    if (count) *count = M;
    if (!x && !cp) return SLLBM_OK;
    if (!ctx->initialised) return fail(ctx, SLLBM_ERR_STATE, "state not initialised");
    cudaSetDevice(ctx->device);
    const int j = side == 0 ? 0 : m.N[1] - 1;
    if (x)
        for (int64_t q = 0; q < M; ++q) {
            const int64_t n = q % m.N[0] + int64_t(m.N[0]) * (j + int64_t(m.N[1]) * (q / m.N[0]));
            for (int d = 0; d < m.D; ++d) x[q * m.D + d] = m.X[size_t(n) * m.D + d];
        }
    if (cp) {
        double *r = nullptr, *u = nullptr, *T = nullptr;
        int rc = moments_on_device(ctx, r, u, T);
        if (rc) return rc;
        if (!ctx->d_cp) CK(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->d_cp), sizeof(double) * M));
        const double denom = 0.5 * ctx->params.gamma * p0 * mach * mach;
        rc = launch_plane_cp(r, T, m.N[0], m.N[1], N2, j, p0, denom, ctx->d_cp, ctx->stream);
        if (rc) return fail(ctx, rc, "pressure coefficient launch failed");
        CK(cudaMemcpyAsync(cp, ctx->d_cp, sizeof(double) * M, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return SLLBM_OK;
}
