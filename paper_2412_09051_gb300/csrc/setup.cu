// FP64 departure-point setup (Sec. 3.1 and Sec. 3.3).
//
// For every arrival node x_AP and velocity zeta_i the departure point is
// x_AP - dt zeta_i (Sec. 3.1).  Axis-aligned meshes locate it per dimension
// (binary search on the cell vertices, periodic wrap); curved O-grid cells are
// inverted by a damped Newton iteration on the isoparametric map while walking
// from the node's home cell towards the point.  A trajectory that leaves the
// domain is cut at its wall point x_W (closed form for the axis-aligned planes,
// 60 bisection steps on curved boundaries) and replaced per Sec. 3.3:
//   equilibrium (3.3.1), bounce-back x_W + iota with iota = zeta_i dt - (x_AP - x_W)
//   reading population ibar (3.3.2), outlet x_AP + zeta_i dt (3.3.3).
// All loops are capped (Newton, walk, bisection); a record that cannot be
// resolved raises an error counter instead of trapping.
#include <cstdio>

#include "sllbm_internal.h"

namespace sllbm {

__device__ __forceinline__ double wrap_periodic(double x, double L) {
    double y = x - L * floor(x / L);
    if (y >= L) y -= L;   // guard against rounding up to L
    if (y < 0) y = 0;
    return y;
}

// --------------------------------------------------------------- axis-aligned
__device__ int locate_axis(const MeshView& M, double x[3], int cc[3], double xr[3], int& bid) {
    bid = -1;
    int inside = 1;
    for (int d = 0; d < M.D; ++d) {
        const double* V = M.V[d];
        const int C = M.cells[d];
        if (M.periodic[d]) {
            x[d] = wrap_periodic(x[d], M.length[d]);
        } else if (x[d] < V[0] || x[d] > V[C]) {
            inside = 0;
            bid = x[d] < V[0] ? 0 : 1;
        }
        // lowest cell c with x <= V[c+1]
        int lo = 0, hi = C - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (x[d] <= V[mid + 1]) hi = mid; else lo = mid + 1;
        }
        cc[d] = lo;
        xr[d] = 2.0 * (x[d] - V[lo]) / (V[lo + 1] - V[lo]) - 1.0;
    }
    return inside;
}

// --------------------------------------------------------------- curved cells
__device__ void lag1d(const MeshView& M, double x, double* L, double* dL) {
    const int p = M.p;
    for (int a = 0; a <= p; ++a) {
        double v = M.glc_inv_den[a];
        double dv = 0.0;
        for (int j = 0; j <= p; ++j) {
            if (j == a) continue;
            double t = M.glc_inv_den[a];
            for (int m = 0; m <= p; ++m)
                if (m != a && m != j) t *= (x - M.glc[m]);
            dv += t;
            v *= (x - M.glc[j]);
        }
        L[a] = v;
        dL[a] = dv;
    }
}

__device__ void naca_map(const MeshView& M, int ca, int cr, const double xi[2], double F[2], double J[2][2]) {
    double La[5], dLa[5], Lb[5], dLb[5];
    lag1d(M, xi[0], La, dLa);
    lag1d(M, xi[1], Lb, dLb);
    F[0] = F[1] = 0.0;
    J[0][0] = J[0][1] = J[1][0] = J[1][1] = 0.0;
    const int p = M.p;
    for (int b = 0; b <= p; ++b)
        for (int a = 0; a <= p; ++a) {
            const int ka = (ca * p + a) % M.N[0];
            const int kb = cr * p + b;
            const double* X = M.X + 2 * (size_t(kb) * M.N[0] + ka);
            const double l = La[a] * Lb[b], da = dLa[a] * Lb[b], db = La[a] * dLb[b];
            for (int d = 0; d < 2; ++d) {
                F[d] += l * X[d];
                J[d][0] += da * X[d];
                J[d][1] += db * X[d];
            }
        }
}

__device__ bool newton_cell(const MeshView& M, int ca, int cr, const double x[2], double xi[2], int max_it) {
    xi[0] = xi[1] = 0.0;
    double F[2], J[2][2];
    for (int it = 0; it < max_it; ++it) {
        naca_map(M, ca, cr, xi, F, J);
        const double r0 = F[0] - x[0], r1 = F[1] - x[1];
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        if (!(fabs(det) > 0.0)) return false;
        double s0 = (J[1][1] * r0 - J[0][1] * r1) / det;
        double s1 = (-J[1][0] * r0 + J[0][0] * r1) / det;
        s0 = fmin(1.0, fmax(-1.0, s0));
        s1 = fmin(1.0, fmax(-1.0, s1));
        xi[0] = fmin(4.0, fmax(-4.0, xi[0] - s0));
        xi[1] = fmin(4.0, fmax(-4.0, xi[1] - s1));
        if (fmax(fabs(s0), fabs(s1)) < 1e-15) break;
        if (it >= 8 && fmax(fabs(xi[0]), fabs(xi[1])) > 2.0) break;
    }
    naca_map(M, ca, cr, xi, F, J);
    return fmax(fabs(F[0] - x[0]), fabs(F[1] - x[1])) < 1e-12;
}

// returns 1 inside (cell/xi set), 0 outside (bid set), -1 walk cap exceeded
__device__ int locate_naca(const TraceArgs& A, const double x[2], int ca0, int cr0, int& cell, double xi[2],
                           int& bid) {
    const MeshView& M = A.M;
    int ca = ca0, cr = cr0;
    const double tol = 1.0 + 1e-12;
    for (int w = 0; w < A.max_walk; ++w) {
        const bool ok = newton_cell(M, ca, cr, x, xi, A.max_newton);
        if (ok && fabs(xi[0]) <= tol && fabs(xi[1]) <= tol) {
            cell = cr * M.cells[0] + ca;
            return 1;
        }
        if (fabs(xi[0]) > tol) {
            ca = (ca + (xi[0] > 0 ? 1 : -1) + M.cells[0]) % M.cells[0];
            continue;
        }
        if (fabs(xi[1]) > tol) {
            const int nr = cr + (xi[1] > 0 ? 1 : -1);
            if (nr < 0) { bid = 0; return 0; }
            if (nr >= M.cells[1]) { bid = 1; return 0; }
            cr = nr;
            continue;
        }
        // Newton did not converge yet ended inside the reference square, which
        // gives no direction (strongly curved cells, e.g. next to the trailing
        // edge at p = 4): search the 3 x 3 neighbourhood and take the lowest
        // containing cell index, the brute-force search's tie rule
        int best = -1;
        double bxi[2] = {0.0, 0.0};
        for (int dr = -1; dr <= 1; ++dr)
            for (int da = -1; da <= 1; ++da) {
                const int r2 = cr + dr, a2 = (ca + da + M.cells[0]) % M.cells[0];
                if ((dr == 0 && da == 0) || r2 < 0 || r2 >= M.cells[1]) continue;
                double xi2[2];
                if (newton_cell(M, a2, r2, x, xi2, A.max_newton) && fabs(xi2[0]) <= tol && fabs(xi2[1]) <= tol) {
                    const int idx = r2 * M.cells[0] + a2;
                    if (best < 0 || idx < best) {
                        best = idx;
                        bxi[0] = xi2[0];
                        bxi[1] = xi2[1];
                    }
                }
            }
        if (best < 0) return -1;
        cell = best;
        xi[0] = bxi[0];
        xi[1] = bxi[1];
        return 1;
    }
    return -1;
}

struct Loc {
    int inside;   // 1 inside, 0 outside, -1 failure
    int cell;
    int bid;
    double xi[3];
    double x[3];  // wrapped point
};

__device__ Loc locate(const TraceArgs& A, const double xin[3], const int home[3]) {
    Loc L;
    L.bid = -1;
    L.cell = -1;
    for (int d = 0; d < 3; ++d) { L.x[d] = xin[d]; L.xi[d] = 0.0; }
    const MeshView& M = A.M;
    if (M.kind != SLLBM_MESH_NACA) {
        int cc[3] = {0, 0, 0};
        L.inside = locate_axis(M, L.x, cc, L.xi, L.bid);
        L.cell = cc[0] + M.cells[0] * (cc[1] + M.cells[1] * cc[2]);
        return L;
    }
    L.inside = locate_naca(A, L.x, home[0], home[1], L.cell, L.xi, L.bid);
    return L;
}

// largest t in [0,1] (to 2^-60) with x0 + t dir inside
__device__ double bisect(const TraceArgs& A, const double x0[3], const double dir[3], const int home[3],
                         double& t_hi, int& bid_hi, int& fail) {
    double lo = 0.0, hi = 1.0;
    bid_hi = -1;
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        double p[3];
        for (int d = 0; d < 3; ++d) p[d] = x0[d] + mid * dir[d];
        Loc L = locate(A, p, home);
        if (L.inside < 0) { fail = 1; }
        if (L.inside == 1) lo = mid; else { hi = mid; bid_hi = L.bid; }
    }
    t_hi = hi;
    return lo;
}

__device__ void trace_one(const TraceArgs& A, int i, const double xap[3], const int home[3], Rec64& r,
                          int& fail) {
    const MeshView& M = A.M;
    const int D = M.D;
    double st[3] = {0, 0, 0}, xdp[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) {
        st[d] = A.dt * A.xi[i][d];
        xdp[d] = xap[d] - st[d];
    }
    Loc L = locate(A, xdp, home);
    if (L.inside < 0) fail = 1;
    int kind = REC_INTERIOR, src = i, bid = 15;
    if (L.inside != 1) {
        double tw, tlo;
        if (M.kind != SLLBM_MESH_NACA) {
            // plane y = V[0] or y = V[C]: closed-form crossing parameter
            const double* V = M.V[1];
            const double yb = xdp[1] < V[0] ? V[0] : V[M.cells[1]];
            bid = xdp[1] < V[0] ? 0 : 1;
            tw = (xap[1] - yb) / st[1];
            tlo = tw;
        } else {
            double thi;
            int bh;
            const double neg[3] = {-st[0], -st[1], -st[2]};
            tlo = bisect(A, xap, neg, home, thi, bh, fail);
            tw = 0.5 * (tlo + thi);
            bid = bh < 0 ? 0 : bh;
        }
        double xw[3] = {0, 0, 0}, xin[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) {
            xw[d] = xap[d] - tw * st[d];
            xin[d] = xap[d] - tlo * st[d];
        }
        if (M.kind != SLLBM_MESH_NACA) {   // keep the start of a clamp segment inside
            const double* V = M.V[1];
            xin[1] = fmin(V[M.cells[1]], fmax(V[0], xin[1]));
        }
        int bk = M.bc_kind[bid];
        if (bk == SLLBM_BC_FARFIELD) bk = xw[0] < 0.5 ? SLLBM_BC_EQUILIBRIUM : SLLBM_BC_OUTLET;
        double xs[3] = {0, 0, 0};
        if (bk == SLLBM_BC_EQUILIBRIUM || bk == SLLBM_BC_PERIODIC) {
            kind = REC_EQ;
            r.cell = -1;
            r.meta = kind | (bid << 4) | (i << 8);
            for (int d = 0; d < 3; ++d) { r.xi[d] = 0.0; r.xsrc[d] = xw[d]; }
            return;
        }
        const double* a;
        if (bk == SLLBM_BC_BOUNCEBACK || bk == SLLBM_BC_ISOTHERMAL) {
            for (int d = 0; d < D; ++d) {
                const double iota = st[d] - (xap[d] - xw[d]);
                xs[d] = xw[d] + iota;
            }
            kind = bk == SLLBM_BC_ISOTHERMAL ? REC_BB_ISO : REC_BB;
            src = A.opp[i];
            a = xin;
        } else {   // outlet: mirrored point
            for (int d = 0; d < D; ++d) xs[d] = xap[d] + st[d];
            kind = REC_OUTLET;
            a = xap;
        }
        L = locate(A, xs, home);
        if (L.inside < 0) fail = 1;
        if (L.inside != 1) {   // the reflected / mirrored point left the domain too: clamp
            double dir[3] = {0, 0, 0}, thi;
            int bh;
            for (int d = 0; d < D; ++d) dir[d] = xs[d] - a[d];
            const double t = bisect(A, a, dir, home, thi, bh, fail);
            for (int d = 0; d < D; ++d) xs[d] = a[d] + t * dir[d];
            L = locate(A, xs, home);
            if (L.inside != 1) fail = 1;
        }
    }
    r.cell = L.cell;
    r.meta = kind | (bid << 4) | (src << 8);
    for (int d = 0; d < 3; ++d) { r.xi[d] = L.xi[d]; r.xsrc[d] = L.x[d]; }
}

// one thread per (unit, velocity); unit = node (gather) or translation class
__global__ void k_trace(TraceArgs A, const double* __restrict__ X, int64_t n_units, int structured,
                        int ncls0, int ncls1, Rec64* __restrict__ out, int* __restrict__ fail_count) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= n_units * A.Q) return;
    const int i = int(t / n_units);
    const int64_t u = t - int64_t(i) * n_units;
    const MeshView& M = A.M;
    int k[3] = {0, 0, 0};
    if (structured) {   // class coordinates are the representative node indices
        k[0] = int(u % ncls0);
        k[1] = int((u / ncls0) % ncls1);
        k[2] = int(u / (int64_t(ncls0) * ncls1));
    } else {
        k[0] = int(u % M.N[0]);
        k[1] = int((u / M.N[0]) % M.N[1]);
        k[2] = int(u / (int64_t(M.N[0]) * M.N[1]));
    }
    const int64_t n = k[0] + int64_t(M.N[0]) * (k[1] + int64_t(M.N[1]) * k[2]);
    double xap[3] = {0, 0, 0};
    for (int d = 0; d < M.D; ++d) xap[d] = X[n * M.D + d];
    int home[3];
    for (int d = 0; d < 3; ++d) home[d] = min(k[d] / M.p, M.cells[d] - 1);
    Rec64 r;
    int fail = 0;
    trace_one(A, i, xap, home, r, fail);
    out[t] = r;
    if (fail) atomicAdd(fail_count, 1);
}

int launch_trace(const TraceArgs& A, const double* dX, int64_t n_units, int structured, int ncls0, int ncls1,
                 Rec64* out, int* d_fail, cudaStream_t s) {
    const int64_t total = n_units * A.Q;
    const int bs = 128;
    const int64_t grid = (total + bs - 1) / bs;
    k_trace<<<unsigned(grid), bs, 0, s>>>(A, dX, n_units, structured, ncls0, ncls1, out, d_fail);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

// per-unit isothermal wall temperature (first velocity hitting an isothermal wall)
__global__ void k_isothermal(const Rec64* __restrict__ rec, int64_t n_units, int Q, const double* __restrict__ bcT,
                             double* __restrict__ Tw, unsigned long long* __restrict__ counts) {
    const int64_t u = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (u >= n_units) return;
    double t = __longlong_as_double(0x7ff8000000000000ULL);
    int nb = 0;
    for (int i = Q - 1; i >= 0; --i) {
        const int meta = rec[int64_t(i) * n_units + u].meta;
        const int kind = meta & 15;
        if (kind != REC_INTERIOR) ++nb;
        if (kind == REC_BB_ISO) t = bcT[(meta >> 4) & 15];
    }
    Tw[u] = t;
    if (nb) atomicAdd(&counts[0], (unsigned long long)nb);
    if (t == t) atomicAdd(&counts[1], 1ULL);
}

int launch_isothermal(const Rec64* rec, int64_t n_units, int Q, const double* bcT, double* Tw,
                      unsigned long long* counts, cudaStream_t s) {
    const int bs = 256;
    k_isothermal<<<unsigned((n_units + bs - 1) / bs), bs, 0, s>>>(rec, n_units, Q, bcT, Tw, counts);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

// gather-mode compact table: code = cell | kind << 24 | bid << 28 (bid 15 none -> 0), xi as real
template <typename real>
__global__ void k_pack_gather(const Rec64* __restrict__ rec, int64_t N, int Q, int D, int32_t* __restrict__ code,
                              real* __restrict__ xi) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= N * Q) return;
    const int i = int(t / N);
    const int64_t n = t - int64_t(i) * N;
    const Rec64 r = rec[t];
    const int kind = r.meta & 15;
    int bid = (r.meta >> 4) & 15;
    if (bid == 15) bid = 0;
    const int cell = r.cell < 0 ? 0 : r.cell;
    code[t] = cell | (kind << 24) | (bid << 28);
    for (int d = 0; d < D; ++d) xi[(int64_t(i) * D + d) * N + n] = real(r.xi[d]);
}

template <typename real>
int launch_pack_gather(const Rec64* rec, int64_t N, int Q, int D, int32_t* code, real* xi, cudaStream_t s) {
    const int bs = 256;
    k_pack_gather<real><<<unsigned((N * Q + bs - 1) / bs), bs, 0, s>>>(rec, N, Q, D, code, xi);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}
template int launch_pack_gather<float>(const Rec64*, int64_t, int, int, int32_t*, float*, cudaStream_t);
template int launch_pack_gather<double>(const Rec64*, int64_t, int, int, int32_t*, double*, cudaStream_t);

}  // namespace sllbm
