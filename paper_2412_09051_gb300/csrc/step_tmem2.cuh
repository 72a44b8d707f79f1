// Fused SLLBM step, row tiles with two arrival nodes per thread: the design of
// step_tmem.cuh (persistent CTAs owning tiles of TY x TZ whole periodic x
// rows, the 2Q streamed values of every node in tensor memory, the source
// rows of each velocity staged once per tile in shared memory) with
//   * one consumer thread per pair of x nodes (x even, x + 1) while
//     streaming: one record (the (y, z) taps are the same for both x
//     parities) and 16-byte tap loads serve two nodes, and the x factor of
//     both comes from a window of six row sums read as three 16-byte loads;
//     two consumer groups take alternate velocities, then every consumer
//     thread collides one node;
//   * one TMA tensor copy per source population and velocity: the union of a
//     tile's (y, z) taps of one population is a box of rows (y range x z
//     range: each row's taps are a product of y and z offsets), copied with
//     cp.async.bulk.tensor over the state viewed as [Q][Nz][Ny][2 NX] FP32
//     (row by row with bulk copies where a box crosses a periodic seam);
//   * stages of up to six consecutive velocities of a group, whose boxes and
//     records one producer warp issues in a single instruction (one lane per
//     copy): the copy engine's cost is per issuing instruction far more than
//     per byte, so few large stages move the rows fastest.
// Tiles of 512 nodes run one CTA per SM; tiles of 256 nodes two, each with
// half of the SM's tensor-memory columns and shared memory, so that one CTA's
// collision overlaps the other's streaming.
// Collision: collide_tmem_pairs for D3Q45 (opposite velocities taken as
// pairs, tensor-memory columns in the pair layout), collide_tmem
// (step_tmem.cuh) for the 2D set.  Every wait is bounded, with the abort
// protocol of step_tmem.cuh.
#pragma once
#include <type_traits>

#include "step_tmem.cuh"

namespace sllbm {

// TMA tensor copy of one box of a 4D tensor (tiled mode) from global to
// shared memory: `tmap` is the generic address of a CUtensorMap in global
// memory, (c0, c1, c2, c3) the box's first element (c0 times the element
// size a multiple of 16 bytes); the bytes count against bar's transaction count
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void* tmap, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ float4 lds4f(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a)
                 : "memory");
    return v;
}
__device__ __forceinline__ int4 lds4(uint32_t a) {
    int4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a)
                 : "memory");
    return v;
}
__device__ __forceinline__ void sts4f(uint32_t a, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// tile class of tile (ty, tz): cy + ncy cz, cy = ty on a non-periodic y axis
// (else ty mod ncy), cz = tz mod ncz
__device__ __forceinline__ int tm2_tile_class(const TmGeom2& T, int ty, int tz, bool py) {
    return (py ? ty % T.ncy : ty) + T.ncy * (tz % T.ncz);
}

// ------------------------------------------------------------ paired collision
// tensor-memory slot of velocity i: the pair layout where the set has one
template <int VS>
__host__ __device__ constexpr int tm2_slot(int i) {
    if constexpr (PairLayout<VS>::on)
        return PairLayout<VS>::slot(i);
    else
        return i;
}
// the D3Q45 slots as a constant table (one uniform load per streamed velocity)
struct Tm2Slots {
    unsigned char s[64];
};
constexpr Tm2Slots tm2_slots45() {
    Tm2Slots t{};
    for (int i = 0; i < VelSet<3>::Q; ++i) t.s[i] = static_cast<unsigned char>(tm2_slot<3>(i));
    return t;
}
static __constant__ Tm2Slots c_tm2_slots45 = tm2_slots45();

// G chunks of 16 FP32 columns of this thread's tensor-memory lane, issued
// together and waited for once (warp-collective)
template <int G>
__device__ __forceinline__ void tm_ld_chunks(uint32_t taddr, float (&v)[16 * G]) {
    static_assert(G == 1 || G == 2, "one or two chunks");
    if constexpr (G == 1) {
        tc_ld16(taddr, v);
    } else {
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr)
            : "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
    }
}

// xi_b . a over the components of base b that are not zero
template <int VS>
__device__ __forceinline__ float pair_dot(const CollideConst<float>& C, int b, float a0, float a1, float a2) {
    using PL = PairLayout<VS>;
    float s = 0.f;
    bool first = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (PL::zero(b) != d) {
            const float a = d == 0 ? a0 : (d == 1 ? a1 : a2);
            s = first ? C.xi[b][d] * a : fmaf(C.xi[b][d], a, s);
            first = false;
        }
    }
    return s;
}

// chunks of 16 columns per tensor-memory load of the paired collision
constexpr int kPairLoadChunks = 1;

// The arithmetic of collide_tmem (moments, isothermal correction, BGK
// relaxation with the quasi-equilibrium heat flux, forcing) for a velocity set
// of opposite pairs, on the pair layout of the node's block: pair k's base
// (f, g) in columns [4k, 4k + 2), its opposite in [4k + 2, 4k + 4), the rest
// velocity in [4 NPAIR, 4 NPAIR + 2).  Each pair is taken at once: with
// c = xi_b . u for the base and -c for the opposite, the equilibrium
// polynomial P1(+-c) = E(c^2) +- c O(c^2) (its even and odd parts); the
// momentum sums take xi_b times the pair's difference.  The heat flux of the
// quasi-equilibrium term comes from moments summed in the same first pass
// (the central third moment of the populations themselves, since the
// equilibrium's vanishes on the set), so the relaxation pass applies the
// correction +-w xi_b . q of g and stores the post-collision pairs: two
// passes over the node state, nothing written back.  Same quantities as
// collide_tmem up to FP32 rounding order.
template <int VS, int GL = kPairLoadChunks>
__device__ __forceinline__ void collide_tmem_pairs(const CollideConst<float>& C, uint32_t tl, float Tw, float2* out,
                                                   int NN, bool store) {
    using VSET = VelSet<VS>;
    using PL = PairLayout<VS>;
    constexpr int NPAIR = PL::NPAIR;
    constexpr int NCH = (4 * NPAIR + 2 + 15) / 16;
    static_assert(VSET::D == 3 && 2 * NPAIR + 1 == VSET::Q, "three-dimensional set of pairs and a rest velocity");
    // ---- moments: plain sums within a chunk (four pairs), Kahan across chunks
    Acc<float> arho, aj0, aj1, aj2, ae;
    // for the heat flux: sum xi_b ((|xi|^2 - (D + 2) - g_f) (f_b - f_o) + g_b - g_o)
    // and the second moments sum xi_a xi_b (f_b + f_o) of the deviations
    float qx0 = 0.f, qx1 = 0.f, qx2 = 0.f, m00 = 0.f, m11 = 0.f, m22 = 0.f, m01 = 0.f, m02 = 0.f, m12 = 0.f;
#pragma unroll
    for (int cg = 0; cg < NCH; cg += GL) {
        float vg[16 * GL];
        tm_ld_chunks<GL>(tl + 16 * cg, vg);
#pragma unroll
        for (int cc = 0; cc < GL; ++cc) {
            const int c = cg + cc;
            float* v = vg + 16 * cc;
            float br = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f, be = 0.f;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int k = 4 * c + m;
                if (k < NPAIR) {
                    const int b = PL::base(k);
                    const float fs = v[4 * m] + v[4 * m + 2], fd = v[4 * m] - v[4 * m + 2];
                    br += fs;
                    if (PL::zero(b) != 0) b0 = fmaf(C.xi[b][0], fd, b0);
                    if (PL::zero(b) != 1) b1 = fmaf(C.xi[b][1], fd, b1);
                    if (PL::zero(b) != 2) b2 = fmaf(C.xi[b][2], fd, b2);
                    be = fmaf(C.s2[VSET::shell(b)], fs, be) + (v[4 * m + 1] + v[4 * m + 3]);
                    {
                        const int z = PL::zero(b);
                        const float tq = fmaf(C.s2[VSET::shell(b)] - 5.f - C.gfac, fd, v[4 * m + 1] - v[4 * m + 3]);
                        if (z != 0) qx0 = fmaf(C.xi[b][0], tq, qx0);
                        if (z != 1) qx1 = fmaf(C.xi[b][1], tq, qx1);
                        if (z != 2) qx2 = fmaf(C.xi[b][2], tq, qx2);
                        if (z != 0) m00 = fmaf(C.xx[b][0], fs, m00);
                        if (z != 1) m11 = fmaf(C.xx[b][1], fs, m11);
                        if (z != 2) m22 = fmaf(C.xx[b][2], fs, m22);
                        if (z != 0 && z != 1) m01 = fmaf(C.xx[b][3], fs, m01);
                        if (z != 0 && z != 2) m02 = fmaf(C.xx[b][4], fs, m02);
                        if (z != 1 && z != 2) m12 = fmaf(C.xx[b][5], fs, m12);
                    }
                } else if (k == NPAIR) {
                    // the rest velocity: xi = 0, |xi|^2 = 0
                    br += v[4 * m];
                    be += v[4 * m + 1];
                }
            }
            arho.add(br);
            aj0.add(b0);
            aj1.add(b1);
            aj2.add(b2);
            ae.add(be);
        }
    }
    const float rho_d = arho.get();
    const float rho = 1.f + rho_d;
    const float inv_rho = 1.f / rho;
    const float u0 = aj0.get() * inv_rho, u1 = aj1.get() * inv_rho, u2 = aj2.get() * inv_rho;
    const float U = u0 * u0 + u1 * u1 + u2 * u2;
    float t = (ae.get() - rho * U - 2.f * C.cv * rho_d) * inv_rho / (2.f * C.cv);
    // The non-equilibrium heat flux sum_i (xi_i - u)(|xi_i - u|^2 f^neq_i +
    // g^neq_i): the equilibrium's central third moment vanishes on the set,
    // so it is the central moment of the node's own populations, written on
    // the deviations with the O(u) parts folded into the sums above (small
    // terms, little FP32 cancellation).  The isothermal correction below
    // changes f and g by equilibria at the same rho and u, which leaves it
    // unchanged.
    const float sc = (5.f + C.gfac) * rho_d - ae.get() + 2.f * rho * U;
    const float qh0 = fmaf(u0, sc, qx0) - 2.f * (m00 * u0 + m01 * u1 + m02 * u2);
    const float qh1 = fmaf(u1, sc, qx1) - 2.f * (m01 * u0 + m11 * u1 + m12 * u2);
    const float qh2 = fmaf(u2, sc, qx2) - 2.f * (m02 * u0 + m12 * u1 + m22 * u2);
    // ---- isothermal wall correction (Eq. thermalBC), on the warps that hold such a node
    const bool iso = !(Tw != Tw);
    if (__any_sync(0xffffffffu, iso)) {
        const float tw = iso ? Tw - 1.f : t;
        const float rT0 = rho * (1.f + t), rT1 = rho * (1.f + tw);
#pragma unroll 1
        for (int c = 0; c < NCH; ++c) {
            float v[16];
            tc_ld16(tl + 16 * c, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int sl = 8 * c + j;   // runtime slot: the per-velocity tables
                if (sl <= 2 * NPAIR) {
                    const int k = sl >> 1;
                    const int i = k == NPAIR ? 0 : ((sl & 1) ? PL::opp(PL::base(k)) : PL::base(k));
                    const float cv = C.xi[i][0] * u0 + C.xi[i][1] * u1 + C.xi[i][2] * u2;
                    const float k2a = 0.5f - 0.25f * U + 0.25f * t * C.sCv[i];
                    const float k1a = 1.0f - 0.5f * U + 0.5f * t * C.sBv[i];
                    const float k0a = -0.5f * U + 0.125f * U * U + 0.5f * t * C.sAv[i] - 0.25f * t * U * C.sBv[i] +
                                      0.125f * t * t * C.sEv[i];
                    const float k2b = 0.5f - 0.25f * U + 0.25f * tw * C.sCv[i];
                    const float k1b = 1.0f - 0.5f * U + 0.5f * tw * C.sBv[i];
                    const float k0b = -0.5f * U + 0.125f * U * U + 0.5f * tw * C.sAv[i] - 0.25f * tw * U * C.sBv[i] +
                                      0.125f * tw * tw * C.sEv[i];
                    const float a0 = eq_poly1(cv, k0a, k1a, k2a), a1 = eq_poly1(cv, k0b, k1b, k2b);
                    if (iso) {
                        v[2 * j] += C.w[i] * rho * (a1 - a0);
                        v[2 * j + 1] += C.wg[i] * ((rT1 * a1 + (rT1 - 1.f)) - (rT0 * a0 + (rT0 - 1.f)));
                    }
                }
            }
            tm_st16(tl + 16 * c, v);
        }
        tm_wait_st();
        if (iso) t = tw;
    }
    const float T = 1.f + t;
    float mu = C.mu_ref;
    if (C.var_mu) mu *= powf(T * C.inv_T_ref, C.mu_exp);
    const float tau = mu / (rho * T * C.dt) + 0.5f;
    const float om = 1.f / tau;
    const float om_pr = 1.f / ((tau - 0.5f) * C.inv_Pr + 0.5f);
    const float rhoT = rho * T;
    const float rhoT_d = rho_d + rho * t;
    // Kupershtokh exact-difference forcing (Sec. 4.3), du = F dt / rho: the
    // equilibrium at v = u + du minus the one at u, added in the relaxation pass
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, V = 0.f;
    if (C.forced) {
        v0 = u0 + C.force_dt[0] * inv_rho;
        v1 = u1 + C.force_dt[1] * inv_rho;
        v2 = u2 + C.force_dt[2] * inv_rho;
        V = v0 * v0 + v1 * v1 + v2 * v2;
    }
    // per-shell coefficients: k0 + k1 c + k2 c^2 + c^3 / 6 + c^4 / 24 at u
    // (and at v), and the weights times rho, rho_d, rho T, rho T_d
    // (the weights are equal within a shell)
    auto rep = [](int sh) { return sh == 0 ? 0 : PL::base(sh == 1 ? 0 : (sh == 2 ? 6 : 16)); };
    float k0[VSET::NS], k1[VSET::NS], k2[VSET::NS], wr[VSET::NS], wrd[VSET::NS], wgr[VSET::NS],
        wgrd[VSET::NS], k0f[VSET::NS], k1f[VSET::NS], k2f[VSET::NS];
#pragma unroll
    for (int sh = 0; sh < VSET::NS; ++sh) {
        k2[sh] = 0.5f - 0.25f * U + 0.25f * t * C.sC[sh];
        k1[sh] = 1.0f - 0.5f * U + 0.5f * t * C.sB[sh];
        k0[sh] = -0.5f * U + 0.125f * U * U + 0.5f * t * C.sA[sh] - 0.25f * t * U * C.sB[sh] +
                 0.125f * t * t * C.sE[sh];
        k2f[sh] = 0.5f - 0.25f * V + 0.25f * t * C.sC[sh];
        k1f[sh] = 1.0f - 0.5f * V + 0.5f * t * C.sB[sh];
        k0f[sh] = -0.5f * V + 0.125f * V * V + 0.5f * t * C.sA[sh] - 0.25f * t * V * C.sB[sh] +
                  0.125f * t * t * C.sE[sh];
        wr[sh] = C.w[rep(sh)] * rho;
        wrd[sh] = C.w[rep(sh)] * rho_d;
        wgr[sh] = C.wg[rep(sh)] * rhoT;
        wgrd[sh] = C.wg[rep(sh)] * rhoT_d;
    }
    // the heat flux relaxes with 1 / tau_Pr: its correction of g, scaled
    const float a = C.quasi ? om - om_pr : 0.f;
    const float q0 = a * qh0, q1 = a * qh1, q2 = a * qh2;
    // ---- relaxation (BGK), the heat-flux correction of g, forcing; the
    // post-collision pairs go to HBM (one pass, nothing written back)
#pragma unroll
    for (int cg = 0; cg < NCH; cg += GL) {
        float vg[16 * GL];
        tm_ld_chunks<GL>(tl + 16 * cg, vg);
#pragma unroll
        for (int cc = 0; cc < GL; ++cc) {
            const int c = cg + cc;
            float* v = vg + 16 * cc;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int k = 4 * c + m;
                if (k < NPAIR) {
                    const int b = PL::base(k), o = PL::opp(b), sh = VSET::shell(b);
                    const float cu = pair_dot<VS>(C, b, u0, u1, u2);
                    const float c2 = cu * cu;
                    const float E = fmaf(c2, fmaf(c2, 1.f / 24.f, k2[sh]), k0[sh]);
                    const float cO = cu * fmaf(c2, 1.f / 6.f, k1[sh]);
                    const float Pb = E + cO, Po = E - cO;
                    const float fb = v[4 * m], gb = v[4 * m + 1], fo = v[4 * m + 2], go = v[4 * m + 3];
                    const float fnb = fb - fmaf(wr[sh], Pb, wrd[sh]), gnb = gb - fmaf(wgr[sh], Pb, wgrd[sh]);
                    const float fno = fo - fmaf(wr[sh], Po, wrd[sh]), gno = go - fmaf(wgr[sh], Po, wgrd[sh]);
                    float rfb = fmaf(-om, fnb, fb), rfo = fmaf(-om, fno, fo);
                    float rgb = fmaf(-om, gnb, gb), rgo = fmaf(-om, gno, go);
                    if (C.forced) {
                        const float cw = pair_dot<VS>(C, b, v0, v1, v2);
                        const float w2 = cw * cw;
                        const float dE = fmaf(w2, fmaf(w2, 1.f / 24.f, k2f[sh]), k0f[sh]) - E;
                        const float dO = fmaf(cw, fmaf(w2, 1.f / 6.f, k1f[sh]), -cO);
                        rfb = fmaf(wr[sh], dE + dO, rfb);
                        rfo = fmaf(wr[sh], dE - dO, rfo);
                    }
                    // the heat-flux correction of g: +- w xi_b . q
                    const float wdq = C.w[b] * pair_dot<VS>(C, b, q0, q1, q2);
                    rgb += wdq;
                    rgo -= wdq;
                    if (store) {
                        out[b * NN] = make_float2(rfb, rgb);
                        out[o * NN] = make_float2(rfo, rgo);
                    }
                } else if (k == NPAIR) {
                    // the rest velocity: c = 0, P1 = k0
                    const float f = v[4 * m], g = v[4 * m + 1];
                    const float fn = f - fmaf(wr[0], k0[0], wrd[0]), gn = g - fmaf(wgr[0], k0[0], wgrd[0]);
                    float rf = fmaf(-om, fn, f);
                    const float rg = fmaf(-om, gn, g);
                    if (C.forced) rf = fmaf(wr[0], k0f[0] - k0[0], rf);
                    if (store) out[0] = make_float2(rf, rg);
                }
            }
        }
    }
}

// Two consumer groups of NX / 2 x TY x TZ threads and one producer warp per
// group.  Group h streams the velocities i = h, h + 2, ... for every pair of
// the tile (thread (row, pair) writes both nodes' values into its tensor-memory
// lane); its producer warp fills the group's own ring of nst / 2 stages, so
// that every stage has one producer and one group of consumers.  After the
// tile's velocities a barrier of all consumers; then thread (h, pair) collides
// node h of its pair (one node per thread).
template <int VS, int NX, int TY, int TZ, int P>
__global__ void __launch_bounds__(NX * TY * TZ + 64, NX * TY * TZ == 512 ? 1 : 2)
    k_step_rows_pairs(const float2* __restrict__ fg, float2* __restrict__ fgo, const void* __restrict__ maps,
                      const int32_t* __restrict__ head, const void* __restrict__ recs,
                      const uint64_t* __restrict__ xmask, const uint64_t* __restrict__ smask,
                      const float* __restrict__ twt, const StepGeom G, const CollideConst<float> C, const TmGeom2 T,
                      int* __restrict__ status) {
    using VSET = VelSet<VS>;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    constexpr int NR = TY * TZ;                   // rows per tile
    constexpr int NP = NX / 2;                    // node pairs per row
    constexpr int NG = NP * NR;                   // threads of one consumer group (one per pair)
    constexpr int NT = 2 * NG;                    // consumer threads
    constexpr int NW = NT / 32;                   // consumer warps
    constexpr int NWG = NW / 2;                   // consumer warps per group
    static_assert(P == 2 || P == 4, "orders 2 and 4");
    using REC = typename std::conditional<P == 2, TmRec2, TmRec4>::type;
    constexpr int XBW = NX;                       // row of the x exchange: slot k holds x = k (periodic)
    constexpr int NXW = 2 * P + 1;                // x weights of a node
    constexpr int REC_BYTES = NR * int(sizeof(REC));        // bytes of one velocity's records (copied)
    // their slot in a stage: a tensor copy's shared-memory destination is
    // 128-byte aligned (stages and row blocks are multiples of 128 bytes)
    constexpr int REC_SLOT = (REC_BYTES + 127) / 128 * 128;
    static_assert((NG == 256 && NW == 16) || (NG == 128 && NW == 8),
                  "two groups of 256 pairs (512 nodes per tile, one CTA per SM) or of 128 pairs (256 nodes per "
                  "tile, two CTAs per SM)");
    constexpr int CPS = NG == 256 ? 1 : 2;        // CTAs per SM
    constexpr int TMA_COLS = TM_ALLOC / CPS;      // tensor-memory columns of this CTA
    static_assert(NP % 32 == 0 && (NP == 32 || 2 * NR <= 14), "whole warps per row; named barriers 1 .. 2 NR");
    static_assert((NP & (NP - 1)) == 0, "pairs of a row a power of two (the exchange indexes modulo NP)");
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    unsigned char* stages = dyn_smem;                                         // [nst][rows | records]
    float2* XB = reinterpret_cast<float2*>(stages + size_t(T.nst) * T.stage_bytes);   // [group][2][NR][XBW]
    uint64_t* bars = reinterpret_cast<uint64_t*>(XB + 4 * NR * XBW);
    // full[nst], empty[nst], and one barrier that nothing completes (waited
    // on only under a test wait limit, so that the timeout path runs)
    uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2 * T.nst + 1);       // TMEM base, abort flag
    volatile int* abort_flag = reinterpret_cast<volatile int*>(slot + 1);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nsh = T.nst / 2;                                                // stages per ring
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8u * uint32_t(T.nst);
    const uint32_t st0 = smem_u32(stages);
    const int NN = int(G.n_nodes);
    const int N1 = G.N[1], N2 = D == 3 ? G.N[2] : 1;
    const bool py = G.periodic[1] != 0;
    const long long lim = wait_limit(status);
    if (tid == 0) {
        for (int s = 0; s < T.nst; ++s) {
            mbar_init(full0 + 8u * uint32_t(s), 1);
            mbar_init(empty0 + 8u * uint32_t(s), NWG);
        }
        mbar_init(full0 + 16u * uint32_t(T.nst), 1);
        *abort_flag = 0;
    }
    if (warp == 0) {
        tc_alloc(smem_u32(slot), TMA_COLS);
        tc_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(slot);
    const int my_tiles = int(blockIdx.x) < T.ntiles ? (T.ntiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;

    if (warp >= NW) {
        // ------------------------------------------------ producer warps
        // Producer h issues the stages of group h (velocities i = h + 2 j)
        // into stages h nst / 2 + (stage count mod nst / 2), all copies of a
        // stage in one instruction: lane 4 q + b the box b of the stage's
        // velocity q, lane 4 TM2_MAX_VEL + q that velocity's records.  The
        // head of its next stage is loaded while the current one is issued.
        const int h = warp - NW;
        const int nv = (Q - h + 1) / 2;                       // velocities of this group
        const int total = my_tiles * nv;
        constexpr int LB = 4 * TM2_MAX_VEL;                   // lanes of the boxes
        static_assert(TM2_MAX_BOXES == 4 && 5 * TM2_MAX_VEL <= 32, "one lane per copy");
        const int q = lane < LB ? (lane >> 2) : lane - LB;    // this lane's velocity in the stage
        const int b = lane & 3;                               // this lane's box
        int s = 0, ph = 0;
        long long seq = 0;
        struct Sd {
            int nvs, bytes, tile, i, n, e, sl, bd;   // velocities, bytes, tile; this lane's velocity, its
        };                                           // boxes, this lane's box, its first slot, its shape
        // all loads of a stage's table entries in one round (none depends on
        // another): this lane's velocity clamped to the group's last, so that
        // every load stays inside the table; the entries beyond the stage or
        // the velocity's boxes are dropped afterwards
        auto fetch = [&](int k) {
            Sd d{1, 0, 0, 0, 0, 0, 0, 0};
            if (k < total) {
                const int kt = k / nv, j0 = k - kt * nv;
                d.tile = int(blockIdx.x) + kt * int(gridDim.x);
                const int tcl = tm2_tile_class(T, d.tile % T.ntile_y, d.tile / T.ntile_y, py);
                const int32_t* h0 = head + (size_t(h + 2 * j0) * T.n_tc + tcl) * TM2_HEAD;
                const int iq = h + 2 * min(j0 + (lane < LB + TM2_MAX_VEL ? q : 0), nv - 1);
                const int32_t* hp = head + (size_t(iq) * T.n_tc + tcl) * TM2_HEAD;
                const int w14 = __ldg(h0 + 14), w15 = __ldg(h0 + 15), n = __ldg(hp);
                const int e = __ldg(hp + 2 + b), sl = __ldg(hp + 2 + TM2_MAX_BOXES + b),
                          bd = __ldg(hp + 2 + 2 * TM2_MAX_BOXES + b);
                d.nvs = max(w14 >> 8, 1);
                d.bytes = w15;
                if (lane < LB + TM2_MAX_VEL && q < d.nvs) {
                    d.i = iq;
                    d.n = n;
                    if (lane < LB && b < n) {
                        d.e = e;
                        d.sl = sl;
                        d.bd = bd;
                    }
                }
            }
            return d;
        };
        Sd da = fetch(0);
#pragma unroll 1
        for (int k = 0; k < total;) {
            const int kn = k + da.nvs;
            const Sd db = fetch(kn);
            const int sg = h * nsh + s;                        // the stage
            if (seq >= nsh) {
                // the stage's previous contents have been read by every warp of the group
                bool ok = !*abort_flag && mbar_wait(empty0 + 8u * uint32_t(sg), uint32_t(ph ^ 1), lim);
                // a consumer that gave up still arrives (after setting the
                // flag): re-read the flag, so that no copy is issued into a
                // stage whose previous copies may still be in flight
                ok = __all_sync(0xffffffffu, ok && !*abort_flag);
                if (!ok) {
                    if (lane == 0) {
                        atomicOr(status, SLLBM_DEV_COPY_TIMEOUT);
                        *abort_flag = 1;
                    }
                    break;
                }
            }
            const uint32_t fb = full0 + 8u * uint32_t(sg);
            const uint32_t sb = st0 + uint32_t(sg) * uint32_t(T.stage_bytes);
            if (lane == 0) mbar_arrive_expect_tx(fb, uint32_t(da.bytes));
            __syncwarp();
            const int ty = da.tile % T.ntile_y, tz = da.tile / T.ntile_y;
            const int y0 = ty * TY, z0 = tz * TZ, tcl = tm2_tile_class(T, ty, tz, py);
            bool act = false, seam = false;
            uint32_t dst = 0;
            int c1 = 0, c2 = 0, c3 = 0, map = 0, by = 0, bz = 0;
            if (lane < LB && q < da.nvs && b < da.n) {
                // a box: population, first y and z (relative to the tile),
                // shape (tensor map); rows [slot, slot + by bz) of the stage
                const int e = da.e;
                c3 = min(e & 63, Q - 1);
                map = (e >> 22) & 63;
                by = da.bd & 255;
                bz = da.bd >> 8;
                c1 = y0 + ((e >> 6) & 255) - 128;
                c2 = D == 3 ? z0 + ((e >> 14) & 255) - 128 : 0;
                dst = sb + uint32_t(da.sl * NX * 8);
                act = c1 >= 0 && c1 + by <= N1 && c2 >= 0 && c2 + bz <= N2;
                seam = !act;
            } else if (lane >= LB && lane < LB + TM2_MAX_VEL && q < da.nvs) {
                // the velocity's records of this tile class: rows [0, NR) of
                // the records tensor [Q][n_tc][NR][32 FP32]
                map = T.rec_map;
                c1 = 0;
                c2 = tcl;
                c3 = da.i;
                dst = sb + uint32_t(T.rows_bytes + q * REC_SLOT);
                act = true;
            }
            if (act && (dst & 127u)) {
                // a tensor copy's shared destination must be 128-byte aligned:
                // record it and skip the copy (the stage's bounded wait then
                // runs out and the step ends with an error)
                atomicOr(status, SLLBM_DEV_BAD_SMEM);
                act = false;
            }
            if (act) tma_load_4d(dst, static_cast<const char*>(maps) + size_t(map) * 128, 0, c1, c2, c3, fb);
            if (seam) {
                // a box across a periodic seam: its rows one z at a time,
                // each y run in one or two pieces (bulk copies)
                for (int dz = 0; dz < bz; ++dz) {
                    int z = c2 + dz;
                    if (D == 3) {
                        z += z < 0 ? N2 : 0;
                        z -= z >= N2 ? N2 : 0;
                    }
                    z = min(max(z, 0), N2 - 1);      // every copy stays inside the mesh
                    const float2* pop = fg + size_t(c3) * NN + size_t(z) * N1 * NX;
                    const uint32_t d = dst + uint32_t(dz * by * NX * 8);
                    int y = c1;
                    if (py) {
                        y += y < 0 ? N1 : 0;
                        y -= y >= N1 ? N1 : 0;
                        y = min(max(y, 0), N1 - 1);
                        const int l1 = min(by, N1 - y);
                        bulk_g2s(d, pop + size_t(y) * NX, uint32_t(l1 * NX * 8), fb);
                        if (by > l1) bulk_g2s(d + uint32_t(l1 * NX * 8), pop, uint32_t((by - l1) * NX * 8), fb);
                    } else {
                        y = min(max(y, 0), N1 - by);
                        bulk_g2s(d, pop + size_t(y) * NX, uint32_t(by * NX * 8), fb);
                    }
                }
            }
            ++seq;
            if (++s == nsh) {
                s = 0;
                ph ^= 1;
            }
            k = kn;
            da = db;
        }
        // on an abort: wait (bounded, default limit) for every copy issued,
        // so that none lands in shared memory after the CTA has exited
        if (*abort_flag && lane == 0) {
            const long long first = seq > nsh ? seq - nsh : 0;
            for (long long u = first; u < seq; ++u)
                mbar_wait(full0 + 8u * uint32_t(h * nsh + int(u % nsh)), uint32_t((u / nsh) & 1));
        }
    } else {
        // ------------------------------------------------ consumers
        // thread (group h, row r, pair xp): nodes x = 2 xp (even) and x + 1
        // (odd); their 2Q values in columns [0, 96) and [96, 192) of a
        // 192-column block of the thread's tensor-memory lane, the same lane
        // and block for both groups (warps w and w + NWG); velocity i in the
        // columns of its slot (the pair layout for D3Q45)
        const int h = tid / NG, pt = tid % NG;
        const int r = pt / NP, xp = pt % NP, x = 2 * xp;
        const int ry = r % TY, rz = r / TY;
        const int nv = (Q - h + 1) / 2;
        const uint32_t tl =
            tbase + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(2 * TM_COLS * ((warp % NWG) >> 2));
        const uint32_t xb0 = smem_u32(XB) + uint32_t((2 * h * NR + r) * XBW * 8);   // this row's halo row, buffer 0
        constexpr uint32_t XBB = uint32_t(NR * XBW * 8);                           // bytes of one buffer
        int s = 0, ph = 0, xb = 0;
        for (int tile = blockIdx.x; tile < T.ntiles; tile += gridDim.x) {
            const int ty = tile % T.ntile_y, tz = tile / T.ntile_y;
            const int y = ty * TY + ry, z = D == 3 ? tz * TZ + rz : 0;
            const bool real = y < N1;
            // velocities whose x factor needs the row exchange, for this tile
            // class: read from global memory, so that every thread of a row
            // takes the same barriers whatever the stage holds
            const int tcl = tm2_tile_class(T, ty, tz, py);
            const uint64_t xm = __ldg(xmask + tcl);
            // velocities of this group that begin a stage
            const uint64_t sm = __ldg(smask + 2 * tcl + h);
            bool live = false;
            int q = 0;
            uint32_t sa = st0;
#pragma unroll 1
            for (int j = 0; j < nv; ++j) {
                const int i = h + 2 * j;
                const int sg = h * nsh + s;
                if ((sm >> j) & 1) {
                    q = 0;
                    sa = st0 + uint32_t(sg) * uint32_t(T.stage_bytes);
                    live = !*abort_flag;
                    // under a test wait limit the first stage also waits on the
                    // barrier that nothing completes (sllbm_debug_wait_limit)
                    if (live && (!mbar_wait(full0 + 8u * uint32_t(sg), uint32_t(ph), lim) ||
                                 (lim < kWaitLimit && j == 0 && !mbar_wait(full0 + 16u * uint32_t(T.nst), 0, lim)))) {
                        atomicOr(status, SLLBM_DEV_COPY_TIMEOUT);
                        *abort_flag = 1;
                        live = false;
                    }
                } else {
                    ++q;
                }
                const uint32_t ra = sa + uint32_t(T.rows_bytes + q * REC_SLOT) + uint32_t(r * int(sizeof(REC)));
                const bool xc = (xm >> i) & 1;
                // after an abort the stage may never have been written: nothing
                // is read from it (an empty equilibrium record instead)
                int meta = REC_EQ;
                float2 sa2 = make_float2(0.f, 0.f), sb2 = make_float2(0.f, 0.f), sa2b = sa2, sb2b = sb2;
                float wxe[NXW], wxo[NXW];
#pragma unroll
                for (int m = 0; m < NXW; ++m) wxe[m] = wxo[m] = 0.f;
                if constexpr (P == 4) {
                    if (live) {
                    // order 4: up to 25 taps; the x weights of this pair's class
                    const REC* R = reinterpret_cast<const REC*>(dyn_smem + (ra - st0));
                    meta = R->meta;
                    const int ntap = R->ntap;
                    if (xc) {
                        const int pc = xp & 1;
#pragma unroll
                        for (int m = 0; m < NXW; ++m) {
                            wxe[m] = reinterpret_cast<const float*>(&R->wx)[(2 * pc) * 9 + m];
                            wxo[m] = reinterpret_cast<const float*>(&R->wx)[(2 * pc + 1) * 9 + m];
                        }
                    }
                    const uint32_t bx = sa + uint32_t(16 * xp);
#pragma unroll
                    for (int k = 0; k < 25; ++k) {
                        if (k < ntap) {
                            const int o = reinterpret_cast<const int32_t*>(&R->off)[k];
                            const float4 v = lds4f(bx + uint32_t(SLLBM_CHK(o, T.rows_bytes, G.status,
                                                                             SLLBM_DEV_BAD_SMEM)));
                            const float wk1 = reinterpret_cast<const float*>(&R->off)[25 + k];
                            const float2 wk = make_float2(wk1, wk1);
                            if (k & 1) {
                                sa2b = __ffma2_rn(wk, make_float2(v.x, v.y), sa2b);
                                sb2b = __ffma2_rn(wk, make_float2(v.z, v.w), sb2b);
                            } else {
                                sa2 = __ffma2_rn(wk, make_float2(v.x, v.y), sa2);
                                sb2 = __ffma2_rn(wk, make_float2(v.z, v.w), sb2);
                            }
                        }
                    }
                    sa2 = __fadd2_rn(sa2, sa2b);
                    sb2 = __fadd2_rn(sb2, sb2b);
                    }
                }
                if constexpr (P == 2) {
                    if (live) {
                    const int4 q0 = lds4(ra), q1 = lds4(ra + 16), q2 = lds4(ra + 32);
                    meta = q0.x;
                    const int ntap = q0.y;
                    if (xc) {
                        const float4 q5 = lds4f(ra + 80), q6 = lds4f(ra + 96), q7 = lds4f(ra + 112);
                        const float wr[10] = {q5.x, q5.y, q5.z, q5.w, q6.x, q6.y, q6.z, q6.w, q7.x, q7.y};
#pragma unroll
                        for (int m = 0; m < NXW; ++m) {
                            wxe[m] = wr[m];
                            wxo[m] = wr[NXW + m];
                        }
                    }
                    if (ntap > 0) {
                        const int4 q3 = lds4(ra + 48), q4 = lds4(ra + 64);
                        const int off[9] = {q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z};
                        const float w[9] = {__int_as_float(q2.w), __int_as_float(q3.x), __int_as_float(q3.y),
                                            __int_as_float(q3.z), __int_as_float(q3.w), __int_as_float(q4.x),
                                            __int_as_float(q4.y), __int_as_float(q4.z), __int_as_float(q4.w)};
                        const uint32_t bx = sa + uint32_t(16 * xp);
                        // both nodes' (f, g) per tap in one 16-byte load; two
                        // accumulators per node (even and odd taps)
                        auto tap = [&](int k) {
                            const float4 v = lds4f(bx + uint32_t(SLLBM_CHK(off[k], T.rows_bytes, G.status,
                                                                             SLLBM_DEV_BAD_SMEM)));
                            const float2 wk = make_float2(w[k], w[k]);
                            if (k & 1) {
                                sa2b = __ffma2_rn(wk, make_float2(v.x, v.y), sa2b);
                                sb2b = __ffma2_rn(wk, make_float2(v.z, v.w), sb2b);
                            } else {
                                sa2 = __ffma2_rn(wk, make_float2(v.x, v.y), sa2);
                                sb2 = __ffma2_rn(wk, make_float2(v.z, v.w), sb2);
                            }
                        };
                        if (ntap == 9) {
#pragma unroll
                            for (int k = 0; k < 9; ++k) tap(k);
                        } else if (ntap == 3) {
#pragma unroll
                            for (int k = 0; k < 3; ++k) tap(k);
                        } else {
#pragma unroll
                            for (int k = 0; k < 9; ++k)
                                if (k < ntap) tap(k);
                        }
                        sa2 = __fadd2_rn(sa2, sa2b);
                        sb2 = __fadd2_rn(sb2, sb2b);
                    }
                    }
                }
                if (j == nv - 1 || ((sm >> (j + 1)) & 1)) {
                    // this warp has read the stage's last velocity: release it to the producer
                    __syncwarp();
                    if (lane == 0) mbar_arrive(empty0 + 8u * uint32_t(sg));
                    if (++s == nsh) {
                        s = 0;
                        ph ^= 1;
                    }
                }
                float2 oa = sa2, ob = sb2;
                if (xc) {
                    // x factor: each node's 2P + 1 x taps among the 2P + 2 row
                    // sums x - P .. x + P + 1, the pairs xp - P / 2 .. xp + P / 2
                    // of the exchange row taken modulo the periodic row
                    const uint32_t xr = xb0 + (xb ? XBB : 0u);
                    sts4f(xr + uint32_t(16 * xp), make_float4(sa2.x, sa2.y, sb2.x, sb2.y));
                    if (NP == 32)
                        __syncwarp();
                    else
                        row_bar(1 + r + h * NR, NP);
                    float2 win[2 * P + 2];
#pragma unroll
                    for (int m = 0; m <= P; ++m) {
                        const float4 wv = lds4f(xr + uint32_t(16 * ((xp + m - P / 2) & (NP - 1))));   // x - P + 2m, + 1
                        win[2 * m] = make_float2(wv.x, wv.y);
                        win[2 * m + 1] = make_float2(wv.z, wv.w);
                    }
                    oa = __fmul2_rn(make_float2(wxe[0], wxe[0]), win[0]);
                    ob = __fmul2_rn(make_float2(wxo[0], wxo[0]), win[1]);
#pragma unroll
                    for (int m = 1; m < NXW; ++m) {
                        oa = __ffma2_rn(make_float2(wxe[m], wxe[m]), win[m], oa);
                        ob = __ffma2_rn(make_float2(wxo[m], wxo[m]), win[m + 1], ob);
                    }
                    xb ^= 1;
                }
                const int kind = meta & 15;
                if (kind != REC_INTERIOR) {
                    const int bid = SLLBM_CHK((meta >> 4) & 15, 2, G.status, SLLBM_DEV_BAD_REC) & 1;
                    if (kind == REC_EQ) {
                        oa = ob = make_float2(C.eqf[bid][i], C.eqg[bid][i]);
                    } else if (kind == REC_BB || kind == REC_BB_ISO) {
                        oa.x += C.mw[bid][i];
                        ob.x += C.mw[bid][i];
                    }
                }
                const int sl = PairLayout<VS>::on ? int(c_tm2_slots45.s[i]) : i;
                tm_st2(tl + 2 * sl, oa.x, oa.y);
                tm_st2(tl + TM_COLS + 2 * sl, ob.x, ob.y);
            }
            // both groups' values of the tile are in tensor memory
            tm_wait_st();
            tc_fence_before();
            row_bar(15, NT);
            tc_fence_after();
            // thread (h, pair) collides node x + h
            const int n = x + h + NX * (y + N1 * z);
            // the node's class: x mod p, y (mod p on a periodic axis), z mod p
            const int cls = (x + h) % P +
                            G.ncls[0] * ((py ? y % P : (real ? y : 0)) + G.ncls[1] * (D == 3 ? z % P : 0));
            const float qnan = __int_as_float(0x7fc00000);
            if constexpr (PairLayout<VS>::on)
                collide_tmem_pairs<VS>(C, tl + uint32_t(h * TM_COLS), real ? __ldg(twt + cls) : qnan, fgo + n, NN,
                                       real && !*abort_flag);
            else
                collide_tmem<VSET>(C, tl + uint32_t(h * TM_COLS), real ? __ldg(twt + cls) : qnan, fgo + n, NN,
                                   real && !*abort_flag);
            // every collision has read its node before the next tile's stores
            tc_fence_before();
            row_bar(15, NT);
            tc_fence_after();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tbase, TMA_COLS);
    }
}

// shared memory of one CTA: the stages, the x-exchange halo rows, the
// barriers, the tensor-memory slot; at least 120 KB for tiles of 512 nodes,
// so that one CTA resides per SM (each allocates all of the SM's
// tensor-memory columns), at least 80 KB for tiles of 256 nodes (two CTAs
// per SM, half of the columns each, never three)
inline size_t rows_pairs_smem_bytes(const TmGeom2& T, int nx, int nr) {
    const size_t b = size_t(T.nst) * T.stage_bytes + sizeof(float2) * 4 * nr * nx +
                     sizeof(uint64_t) * (2 * T.nst + 1) + 16;
    const size_t lo = nx * nr == 512 ? 120 * 1024 : 80 * 1024;
    return b < lo ? lo : b;
}

template <int VS, int NX, int TY, int TZ, int P>
int launch_step_rows_pairs(const float2* fg, float2* fgo, const void* maps, const int32_t* head, const void* recs,
                           const uint64_t* xmask, const uint64_t* smask, const float* tw, const StepGeom& G,
                           const CollideConst<float>& C, const TmGeom2& T, int* status, cudaStream_t stream, int grid) {
    const size_t smem = rows_pairs_smem_bytes(T, NX, TY * TZ);
    if (cudaFuncSetAttribute(k_step_rows_pairs<VS, NX, TY, TZ, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem)) != cudaSuccess)
        return SLLBM_ERR_CUDA;
    k_step_rows_pairs<VS, NX, TY, TZ, P><<<grid, NX * TY * TZ + 64, smem, stream>>>(fg, fgo, maps, head, recs, xmask,
                                                                                    smask, tw, G, C, T, status);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

}  // namespace sllbm
