// Device-side building blocks of the fused SLLBM step.
//
// Equilibrium (Sec. 3.1, order-4 Hermite expansion, Shan et al. 2006 form):
// with c = xi_i . u, s = |xi_i|^2, U = |u|^2, t = T - 1 (T0 = 1) the
// contraction sum_n a^(n) : H^(n)_i / n! collapses to the scalar polynomial
//   P_i = 1 + c + c^2/2 + c^3/6 + c^4/24
//           + c^2 (-U/4 + t C/4) + c (-U/2 + t B/2)
//           + (-U/2 + U^2/8 + t A/2 - t U B/4 + t^2 E/8)
// where A = s - D, B = s - D - 2, C = s - D - 4, E = s^2 - 2(D+2)s + D(D+2)
// depend only on the velocity shell.  f_i^eq = w_i rho P_i and
// g_i^eq = T (2 c_v - D) f_i^eq.  Populations are carried as deviations
// from the reference values w_i (f) and w_i (2 c_v - D) (g).
#pragma once
#include <cmath>
#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#define SLLBM_QMAX 45
#define SLLBM_SMAX 6

namespace sllbm {

template <typename real> struct Vec2;
template <> struct Vec2<float> {
    using T = float2;
    __host__ __device__ static float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct Vec2<double> {
    using T = double2;
    __host__ __device__ static double2 make(double a, double b) { return make_double2(a, b); }
};

// ------------------------------------------------------------ velocity sets
// Compile-time structure (Q, D, shell of each index); numeric values arrive
// at run time in CollideConst.
template <int VS> struct VelSet;

template <> struct VelSet<0> {   // D2Q9
    static constexpr int Q = 9, D = 2, NS = 3;
    __host__ __device__ static constexpr int shell(int i) {
        return i == 0 ? 0 : ((i == 1 || i == 2 || i == 5 || i == 6) ? 1 : 2);
    }
};
template <> struct VelSet<1> {   // D2Q19
    static constexpr int Q = 19, D = 2, NS = 4;
    __host__ __device__ static constexpr int shell(int i) { return i == 0 ? 0 : 1 + (i - 1) / 6; }
};
template <> struct VelSet<2> {   // D2Q25
    static constexpr int Q = 25, D = 2, NS = 6;
    __host__ __device__ static constexpr int cls(int a) { return a == 0 ? 0 : ((a == 1 || a == 3) ? 1 : 2); }
    __host__ __device__ static constexpr int shell(int i) {
        // unordered pair of 1D node classes -> 0..5
        return (cls(i % 5) <= cls(i / 5))
                   ? (cls(i % 5) == 0 ? cls(i / 5) : (cls(i % 5) == 1 ? 2 + cls(i / 5) : 5))
                   : (cls(i / 5) == 0 ? cls(i % 5) : (cls(i / 5) == 1 ? 2 + cls(i % 5) : 5));
    }
};
template <> struct VelSet<3> {   // D3Q45
    static constexpr int Q = 45, D = 3, NS = 4;
    __host__ __device__ static constexpr int shell(int i) {
        return i == 0 ? 0 : (i <= 12 ? 1 : (i <= 32 ? 2 : 3));
    }
};

// Opposite pairs of a velocity set (xi_o = -xi_b, w_o = w_b), for the paired
// collision: pair k = (base(k), opp(base(k))); zero(b) is the component that
// is zero in both (-1: none); slot(i) places pair k at slots 2k (base) and
// 2k + 1 (opposite) and the rest velocity at slot 2 NPAIR.  The host checks
// the numeric table against this structure before a kernel relies on it.
template <int VS> struct PairLayout {
    static constexpr bool on = false;
};
template <> struct PairLayout<3> {   // D3Q45: icosahedron, dodecahedron, icosahedron shells
    static constexpr bool on = true;
    static constexpr int NPAIR = 22;
    // bases 1..6 (shell 1), 13..22 (shell 2), 33..38 (shell 3)
    __host__ __device__ static constexpr int base(int k) { return k < 6 ? 1 + k : (k < 16 ? 7 + k : 17 + k); }
    __host__ __device__ static constexpr int opp(int b) { return b + ((b >= 13 && b <= 22) ? 10 : 6); }
    // the cyclic (0, a, b) patterns: x, y, z zero in consecutive index pairs;
    // 13..16 are the (+-1, +-1, +-1) directions
    __host__ __device__ static constexpr int zero(int b) {
        return b <= 12 ? (b - 1) / 2 : (b <= 16 ? -1 : (b <= 32 ? (b - 17) / 2 : (b - 33) / 2));
    }
    __host__ __device__ static constexpr int slot(int i) {
        return i == 0    ? 2 * NPAIR
               : i <= 6  ? 2 * (i - 1)
               : i <= 12 ? 2 * (i - 7) + 1
               : i <= 22 ? 2 * (i - 7)
               : i <= 32 ? 2 * (i - 17) + 1
               : i <= 38 ? 2 * (i - 17)
                         : 2 * (i - 23) + 1;
    }
};

// ------------------------------------------------------------ constants
template <typename real>
struct CollideConst {
    real xi[SLLBM_QMAX][3];
    real w[SLLBM_QMAX];
    real wg[SLLBM_QMAX];          // w_i (2 c_v - D)
    real sA[SLLBM_SMAX], sB[SLLBM_SMAX], sC[SLLBM_SMAX], sE[SLLBM_SMAX], s2[SLLBM_SMAX];
    real cv, gfac;                // c_v and (2 c_v - D)
    real dt, inv_Pr;
    real mu_ref, inv_T_ref, mu_exp;
    int  var_mu;                  // mu_exp != 0
    int  quasi;                   // Pr != 1
    int  forced;                  // body force present
    real force_dt[3];             // F dt (force density times time step)
    // boundary constants per boundary id: equilibrium deviations and moving-wall term
    real eqf[2][SLLBM_QMAX];
    real eqg[2][SLLBM_QMAX];
    real mw[2][SLLBM_QMAX];
    int opp[SLLBM_QMAX];
    // per-velocity copies of the shell constants (runtime-indexed loops)
    real s2v[SLLBM_QMAX], sAv[SLLBM_QMAX], sBv[SLLBM_QMAX], sCv[SLLBM_QMAX], sEv[SLLBM_QMAX];
    // second-moment products xi_a xi_b per velocity: (00, 11, 22, 01, 02, 12)
    real xx[SLLBM_QMAX][6];
};

// ------------------------------------------------------------ compensated sum
template <typename real>
struct Acc {
    real s, c;
    __device__ __forceinline__ Acc() : s(0), c(0) {}
    __device__ __forceinline__ void add(real x) { s += x; }
    __device__ __forceinline__ real get() const { return s; }
};
template <>
struct Acc<float> {   // Kahan summation (no fast-math: the compensation survives)
    float s, c;
    __device__ __forceinline__ Acc() : s(0.f), c(0.f) {}
    __device__ __forceinline__ void add(float x) {
        float y = __fsub_rn(x, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ float get() const { return s; }
};

// ------------------------------------------------------------ equilibrium
// Shell coefficients of P_i - 1 = ((c/24 + 1/6) c + k2) c^2 ... evaluated as
// P1 = (((c * (1/24) + 1/6) * c + k2) * c + k1) * c + k0.
template <typename real, int NS>
struct EqCoef {
    real k0[NS], k1[NS], k2[NS];
    __device__ __forceinline__ void build(const CollideConst<real>& C, real U, real t) {
        const real tU = t * U;
        const real t2 = t * t;
#pragma unroll
        for (int h = 0; h < NS; ++h) {
            k2[h] = real(0.5) - real(0.25) * U + real(0.25) * t * C.sC[h];
            k1[h] = real(1.0) - real(0.5) * U + real(0.5) * t * C.sB[h];
            k0[h] = -real(0.5) * U + real(0.125) * U * U + real(0.5) * t * C.sA[h]
                    - real(0.25) * tU * C.sB[h] + real(0.125) * t2 * C.sE[h];
        }
    }
};

template <typename real>
__device__ __forceinline__ real eq_poly1(real c, real k0, real k1, real k2) {
    return (((c * real(1.0 / 24.0) + real(1.0 / 6.0)) * c + k2) * c + k1) * c + k0;
}

// f^eq and g^eq deviations of one velocity for the node state (rho, u, T):
//   fdev = w (rho P1 + (rho - 1)),  gdev = wg (rho T P1 + (rho T - 1))
template <class VSET, typename real, int I>
__device__ __forceinline__ void eq_dev(const CollideConst<real>& C, const EqCoef<real, VSET::NS>& K,
                                       const real (&u)[3], real rho, real rho_d, real rhoT, real rhoT_d,
                                       real& fdev, real& gdev, real& cdot) {
    constexpr int h = VSET::shell(I);
    real c = C.xi[I][0] * u[0] + C.xi[I][1] * u[1];
    if (VSET::D == 3) c += C.xi[I][2] * u[2];
    const real P1 = eq_poly1(c, K.k0[h], K.k1[h], K.k2[h]);
    fdev = C.w[I] * (rho * P1 + rho_d);
    gdev = C.wg[I] * (rhoT * P1 + rhoT_d);
    cdot = c;
}

template <int I, int N>
struct Unroll {
    template <class F>
    __device__ __forceinline__ static void run(F&& f) {
        f(std::integral_constant<int, I>());
        Unroll<I + 1, N>::run(f);
    }
};
template <int N>
struct Unroll<N, N> {
    template <class F>
    __device__ __forceinline__ static void run(F&&) {}
};

// ------------------------------------------------------------ collide
// In: streamed deviations f[Q], g[Q]; Tw = wall temperature of the node's
// isothermal correction (Eq. thermalBC) or NaN.  Out: post-collision
// deviations (Eq. 1).  Returns the node density (for diagnostics).
template <class VSET, typename real>
__device__ __forceinline__ void collide_node(const CollideConst<real>& C, real (&f)[VSET::Q],
                                             real (&g)[VSET::Q], real Tw, real* fneq = nullptr) {
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    // ---- moments (compensated in FP32)
    Acc<real> arho, aj0, aj1, aj2, ae;
    Unroll<0, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        arho.add(f[i]);
        aj0.add(C.xi[i][0] * f[i]);
        aj1.add(C.xi[i][1] * f[i]);
        if (D == 3) aj2.add(C.xi[i][2] * f[i]);
        ae.add(C.s2[VSET::shell(i)] * f[i]);
        ae.add(g[i]);
    });
    const real rho_d = arho.get();
    const real rho = real(1) + rho_d;
    const real inv_rho = real(1) / rho;
    real u[3] = {aj0.get() * inv_rho, aj1.get() * inv_rho, D == 3 ? aj2.get() * inv_rho : real(0)};
    const real U = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    // 2 rho c_v T = e + 2 c_v - rho U  ->  t = T - 1 = (e - rho U - 2 c_v rho_d) / (2 rho c_v)
    real t = (ae.get() - rho * U - real(2) * C.cv * rho_d) * inv_rho / (real(2) * C.cv);

    // ---- isothermal wall correction (Eq. thermalBC): f += f^eq(T_w) - f^eq(T)
    if (!(Tw != Tw)) {
        const real tw = Tw - real(1);
        EqCoef<real, VSET::NS> K0, K1;
        K0.build(C, U, t);
        K1.build(C, U, tw);
        const real rhoT0 = rho * (real(1) + t), rhoT1 = rho * (real(1) + tw);
        Unroll<0, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            real f0, g0, f1, g1, cd;
            eq_dev<VSET, real, i>(C, K0, u, rho, rho_d, rhoT0, rhoT0 - real(1), f0, g0, cd);
            eq_dev<VSET, real, i>(C, K1, u, rho, rho_d, rhoT1, rhoT1 - real(1), f1, g1, cd);
            f[i] += f1 - f0;
            g[i] += g1 - g0;
        });
        t = tw;
    }
    const real T = real(1) + t;
    // ---- relaxation times (tau = mu / (p dt) + 1/2, tau_Pr = (tau - 1/2)/Pr + 1/2)
    real mu = C.mu_ref;
    if (C.var_mu) mu *= pow(T * C.inv_T_ref, C.mu_exp);
    const real tau = mu / (rho * T * C.dt) + real(0.5);
    const real om = real(1) / tau;
    const real om_pr = real(1) / ((tau - real(0.5)) * C.inv_Pr + real(0.5));

    EqCoef<real, VSET::NS> K;
    K.build(C, U, t);
    const real rhoT = rho * T;
    const real rhoT_d = rho_d + rho * t;
    real q0 = 0, q1 = 0, q2 = 0;
    Unroll<0, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        real fe, ge, cd;
        eq_dev<VSET, real, i>(C, K, u, rho, rho_d, rhoT, rhoT_d, fe, ge, cd);
        const real fn = f[i] - fe;
        const real gn = g[i] - ge;
        if (fneq) fneq[i] = fn;
        // central heat flux (times 2): sum (xi - u) (|xi - u|^2 f^neq + g^neq)
        const real cu2 = C.s2[VSET::shell(i)] - real(2) * cd + U;
        const real h = cu2 * fn + gn;
        q0 += (C.xi[i][0] - u[0]) * h;
        q1 += (C.xi[i][1] - u[1]) * h;
        if (D == 3) q2 += (C.xi[i][2] - u[2]) * h;
        f[i] -= om * fn;
        g[i] -= om * gn;
    });
    if (C.quasi) {
        // g*_i = w_i xi_i . (2 q^neq), weighted by (1/tau - 1/tau_Pr)
        const real a = om - om_pr;
        q0 *= a;
        q1 *= a;
        q2 *= a;
        Unroll<0, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            real d = C.xi[i][0] * q0 + C.xi[i][1] * q1;
            if (D == 3) d += C.xi[i][2] * q2;
            g[i] += C.w[i] * d;
        });
    }
    if (C.forced) {
        // Kupershtokh exact-difference forcing (Sec. 4.3):
        // f_i += f_i^eq(rho, u + du, T) - f_i^eq(rho, u, T), du = F dt / rho
        real v[3] = {u[0] + C.force_dt[0] * inv_rho, u[1] + C.force_dt[1] * inv_rho,
                     D == 3 ? u[2] + C.force_dt[2] * inv_rho : real(0)};
        const real V = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        EqCoef<real, VSET::NS> K1;
        K1.build(C, V, t);
        Unroll<0, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            real fa, ga, fb, gb, cd;
            eq_dev<VSET, real, i>(C, K1, v, rho, rho_d, rhoT, rhoT_d, fa, ga, cd);
            eq_dev<VSET, real, i>(C, K, u, rho, rho_d, rhoT, rhoT_d, fb, gb, cd);
            f[i] += fa - fb;
        });
    }
}

// ------------------------------------------------------------ Lagrange basis
// 1D Lagrange polynomials of order P on the GLC nodes at x (nodes / inverse
// denominators supplied by the caller).
template <int P, typename real>
__device__ __forceinline__ void lagrange_w(real x, const real* xh, const real* inv_den, real (&L)[P + 1]) {
#pragma unroll
    for (int a = 0; a <= P; ++a) {
        real v = inv_den[a];
#pragma unroll
        for (int m = 0; m <= P; ++m)
            if (m != a) v *= (x - xh[m]);
        L[a] = v;
    }
}

}  // namespace sllbm

namespace sllbm {

// ------------------------------------------------------------ collide, state in shared memory
// Same arithmetic as collide_node with runtime velocity loops: the streamed
// deviations of the thread's node sit at Sf[i * stride], Sg[i * stride]; the
// post-collision pair of velocity i is written to out[i * NN] (out == nullptr:
// no store).
// KEEP: the post-collision pair stays in Sf / Sg (quasi-equilibrium and
// forcing applied in place) and f^neq of the streamed state goes to Sn; out is
// not used (the learned correction is added before the store).
template <class VSET, typename real, typename V2, int stride, bool KEEP = false>
__device__ __forceinline__ void collide_smem(const CollideConst<real>& C, real* Sf, real* Sg, real Tw,
                                             V2* out, int NN, real* Sn = nullptr) {
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    // blocked compensation: plain sums over groups of 5 velocities, the
    // group sums added with Kahan's compensation (error ~5 eps max|f| per sum
    // instead of ~2 eps, at a fifth of the compensation cost); a runtime loop
    // over the groups keeps the body small for the instruction cache
    Acc<real> arho, aj0, aj1, aj2, ae;
    constexpr int B = 5;
#pragma unroll 1
    for (int i0 = 0; i0 < Q; i0 += B) {
        real br = 0, b0 = 0, b1 = 0, b2 = 0, be = 0;
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int i = i0 + k;
            if (i < Q) {
                const real f = Sf[i * stride], g = Sg[i * stride];
                br += f;
                b0 += C.xi[i][0] * f;
                b1 += C.xi[i][1] * f;
                if (D == 3) b2 += C.xi[i][2] * f;
                be += C.s2v[i] * f + g;
            }
        }
        arho.add(br);
        aj0.add(b0);
        aj1.add(b1);
        if (D == 3) aj2.add(b2);
        ae.add(be);
    }
    const real rho_d = arho.get();
    const real rho = real(1) + rho_d;
    const real inv_rho = real(1) / rho;
    const real u0 = aj0.get() * inv_rho, u1 = aj1.get() * inv_rho, u2 = D == 3 ? aj2.get() * inv_rho : real(0);
    const real U = u0 * u0 + u1 * u1 + u2 * u2;
    real t = (ae.get() - rho * U - real(2) * C.cv * rho_d) * inv_rho / (real(2) * C.cv);
    // P1 of velocity i for temperature offset tt
    auto p1 = [&](int i, real tt, real& cd) {
        real c = C.xi[i][0] * u0 + C.xi[i][1] * u1;
        if (D == 3) c += C.xi[i][2] * u2;
        cd = c;
        // per-shell coefficients: in the unrolled loops the shell is a
        // compile-time index, so velocities of one shell share k0, k1, k2
        const int sh = VSET::shell(i);
        const real k2 = real(0.5) - real(0.25) * U + real(0.25) * tt * C.sC[sh];
        const real k1 = real(1.0) - real(0.5) * U + real(0.5) * tt * C.sB[sh];
        const real k0 = -real(0.5) * U + real(0.125) * U * U + real(0.5) * tt * C.sA[sh] -
                        real(0.25) * tt * U * C.sB[sh] + real(0.125) * tt * tt * C.sE[sh];
        return eq_poly1(c, k0, k1, k2);
    };
    if (!(Tw != Tw)) {   // isothermal wall correction (Eq. thermalBC)
        const real tw = Tw - real(1);
        const real rT0 = rho * (real(1) + t), rT1 = rho * (real(1) + tw);
        // runtime loop: only nodes next to an isothermal wall take this
        // branch, and a compact body keeps it out of the instruction cache's
        // way on every other node
#pragma unroll 1
        for (int i = 0; i < Q; ++i) {
            real cd;
            const real a0 = p1(i, t, cd), a1 = p1(i, tw, cd);
            Sf[i * stride] += C.w[i] * rho * (a1 - a0);
            Sg[i * stride] += C.wg[i] * ((rT1 * a1 + (rT1 - real(1))) - (rT0 * a0 + (rT0 - real(1))));
        }
        t = tw;
    }
    const real T = real(1) + t;
    real mu = C.mu_ref;
    if (C.var_mu) mu *= pow(T * C.inv_T_ref, C.mu_exp);
    const real tau = mu / (rho * T * C.dt) + real(0.5);
    const real om = real(1) / tau;
    const real om_pr = real(1) / ((tau - real(0.5)) * C.inv_Pr + real(0.5));
    const real rhoT = rho * T;
    const real rhoT_d = rho_d + rho * t;
    real q0 = 0, q1 = 0, q2 = 0;
    // BGK relaxation of velocity i; accumulates the heat flux of the
    // quasi-equilibrium term
    auto relax = [&](int i, real& fo, real& go, real& fno) {
        real cd;
        const real P1 = p1(i, t, cd);
        const real fe = C.w[i] * (rho * P1 + rho_d);
        const real ge = C.wg[i] * (rhoT * P1 + rhoT_d);
        const real f = Sf[i * stride], g = Sg[i * stride];
        const real fn = f - fe, gn = g - ge;
        const real h = (C.s2v[i] - real(2) * cd + U) * fn + gn;
        q0 += (C.xi[i][0] - u0) * h;
        q1 += (C.xi[i][1] - u1) * h;
        if (D == 3) q2 += (C.xi[i][2] - u2) * h;
        fo = f - om * fn;
        go = g - om * gn;
        fno = fn;
    };
    // one loop per destination, chosen once: a per-velocity test in the
    // unrolled loop costs instruction fetch on every node
    if (KEEP) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            real fo, go, fn;
            relax(i, fo, go, fn);
            Sf[i * stride] = fo;
            Sg[i * stride] = go;
            Sn[i * stride] = fn;
        }
    } else if (C.quasi || C.forced) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            real fo, go, fn;
            relax(i, fo, go, fn);
            Sf[i * stride] = fo;
            Sg[i * stride] = go;
        }
    } else if (out) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            real fo, go, fn;
            relax(i, fo, go, fn);
            out[i * NN] = Vec2<real>::make(fo, go);
        }
    }
    if (KEEP && (C.quasi || C.forced)) {
        const real a = om - om_pr;
        q0 *= C.quasi ? a : real(0);
        q1 *= C.quasi ? a : real(0);
        q2 *= C.quasi ? a : real(0);
        const real v0 = u0 + C.force_dt[0] * inv_rho, v1 = u1 + C.force_dt[1] * inv_rho;
        const real v2 = D == 3 ? u2 + C.force_dt[2] * inv_rho : real(0);
        const real V = v0 * v0 + v1 * v1 + v2 * v2;
#pragma unroll 1
        for (int i = 0; i < Q; ++i) {
            real dq = C.xi[i][0] * q0 + C.xi[i][1] * q1;
            if (D == 3) dq += C.xi[i][2] * q2;
            Sg[i * stride] += C.w[i] * dq;
            if (C.forced) {   // Kupershtokh exact-difference forcing (Sec. 4.3)
                real cd;
                const real pa = p1(i, t, cd);
                real c = C.xi[i][0] * v0 + C.xi[i][1] * v1;
                if (D == 3) c += C.xi[i][2] * v2;
                const real k2 = real(0.5) - real(0.25) * V + real(0.25) * t * C.sCv[i];
                const real k1 = real(1.0) - real(0.5) * V + real(0.5) * t * C.sBv[i];
                const real k0 = -real(0.5) * V + real(0.125) * V * V + real(0.5) * t * C.sAv[i] -
                                real(0.25) * t * V * C.sBv[i] + real(0.125) * t * t * C.sEv[i];
                Sf[i * stride] += C.w[i] * rho * (eq_poly1(c, k0, k1, k2) - pa);
            }
        }
    }
    if (!KEEP && (C.quasi || C.forced)) {
        const real a = om - om_pr;
        q0 *= C.quasi ? a : real(0);
        q1 *= C.quasi ? a : real(0);
        q2 *= C.quasi ? a : real(0);
        // Kupershtokh exact-difference forcing (Sec. 4.3), du = F dt / rho
        const real v0 = u0 + C.force_dt[0] * inv_rho, v1 = u1 + C.force_dt[1] * inv_rho;
        const real v2 = D == 3 ? u2 + C.force_dt[2] * inv_rho : real(0);
        const real V = v0 * v0 + v1 * v1 + v2 * v2;
        // the forcing test is hoisted out of the unrolled loop: interleaved
        // with it, the never-taken forcing code filled the instruction cache
        // lines of the quasi-equilibrium pass
        if (out && !C.forced) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                real dq = C.xi[i][0] * q0 + C.xi[i][1] * q1;
                if (D == 3) dq += C.xi[i][2] * q2;
                out[i * NN] = Vec2<real>::make(Sf[i * stride], Sg[i * stride] + C.w[i] * dq);
            }
        } else if (out) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                real dq = C.xi[i][0] * q0 + C.xi[i][1] * q1;
                if (D == 3) dq += C.xi[i][2] * q2;
                real fo = Sf[i * stride];
                if (C.forced) {
                    real cd;
                    const real pa = p1(i, t, cd);
                    real c = C.xi[i][0] * v0 + C.xi[i][1] * v1;
                    if (D == 3) c += C.xi[i][2] * v2;
                    const real k2 = real(0.5) - real(0.25) * V + real(0.25) * t * C.sCv[i];
                    const real k1 = real(1.0) - real(0.5) * V + real(0.5) * t * C.sBv[i];
                    const real k0 = -real(0.5) * V + real(0.125) * V * V + real(0.5) * t * C.sAv[i] -
                                    real(0.25) * t * V * C.sBv[i] + real(0.125) * t * t * C.sEv[i];
                    fo += C.w[i] * rho * (eq_poly1(c, k0, k1, k2) - pa);
                }
                out[i * NN] = Vec2<real>::make(fo, Sg[i * stride] + C.w[i] * dq);
            }
        }
    }
}

}  // namespace sllbm
