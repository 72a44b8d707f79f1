// Fused SLLBM step for axis-aligned meshes with a periodic x axis: a
// persistent kernel whose CTAs own tiles of TY x TZ whole x rows (TY x TZ x NX
// arrival nodes, one per thread), with the node state held in tensor memory
// and all of shared memory given to a pipeline of source rows.
//
// Streaming (Sec. 3.1, streamed-value formula): on these meshes the departure
// cell of velocity i depends on the arrival node only through its class
// (x parity, y index, z parity), and its Lagrange weights factorise into x and
// (y, z) parts.  For one velocity, a tile needs a short list of whole source
// rows (population, y', z'): the union of the (y, z) taps of its rows, each
// row NX contiguous (f, g) pairs, merged into runs of consecutive y rows per
// (population, z) that are contiguous in memory.  Two producer warps, taking
// alternate velocities, copy the runs with the TMA bulk-copy engine
// (cp.async.bulk, completion on the stage's mbarrier), up to nst velocities
// ahead, together with the tile's per-row records; the consumer
// threads contract the (y, z) taps from shared memory, exchange the row sums
// of their x row through a small halo buffer (one named barrier per row and
// velocity) for the three x taps, and store the streamed (f, g) pair of every
// velocity into two columns of their tensor-memory lane (tcgen05.st).
// Rows are read from HBM once per tile instead of once per arrival row and
// tap, and every source row copied serves all rows of the tile.
//
// Collision (Sec. 3.1 Eq. 1 with the boundary terms of Sec. 3.3): the node's
// 2Q values come back from tensor memory in chunks of 16 columns
// (tcgen05.ld) for the compensated moment sums, the isothermal-wall
// correction (Eq. thermalBC), the BGK relaxation with the quasi-equilibrium
// heat-flux term and the Kupershtokh forcing; the post-collision pairs are
// stored to HBM.
//
// Every wait is bounded: a wait that runs out records SLLBM_DEV_COPY_TIMEOUT
// in the status word, sets the CTA's abort flag (after which no thread waits
// again), the producer waits (bounded) for the copies it issued, and the CTA
// frees its tensor memory and exits.
#pragma once
#include "bulk.cuh"
#include "checked.cuh"
#include "mlp_tc.cuh"
#include "sllbm_internal.h"

namespace sllbm {

__device__ __forceinline__ void tm_st2(uint32_t taddr, float a, float b) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(__float_as_uint(a)),
                 "r"(__float_as_uint(b))
                 : "memory");
}
__device__ __forceinline__ void tm_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// one FP32 column of this thread's TMEM lane (warp-collective; waits)
__device__ __forceinline__ float tm_ld1(uint32_t taddr) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=r"(r)
                 : "r"(taddr)
                 : "memory");
    return __uint_as_float(r);
}
// FP32 rounded to TF32 (cvt.rna: nearest, ties away from zero), in an FP32 container
__device__ __forceinline__ float to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}
__device__ __forceinline__ void sts1(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ float2 lds2_tm(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
// tcgen05.mma of kind::tf32: D (TMEM) += A (smem) . B (smem)^T
__device__ __forceinline__ void tc_mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
// byte offset of element (r, k) of an R x K TF32 operand in the canonical
// K-major layout without swizzle (8 x 16-byte core matrices, 128 B apart
// along K, K * 32 B apart along R)
__device__ __forceinline__ uint32_t tf32_canon(int r, int k, int K) {
    return uint32_t((r >> 3) * (K * 32) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// barrier over the `count` threads of one x row (ids 1 .. TY TZ; 0 is
// __syncthreads); rows of one warp synchronise with __syncwarp instead
__device__ __forceinline__ void row_bar(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// ------------------------------------------------------------ collision from tensor memory
// The arithmetic of collide_smem (blocked compensated moments, isothermal
// correction, relaxation with the heat-flux quasi-equilibrium term, forcing)
// on the 2Q values of this thread's node in columns [2i, 2i + 1] of its
// tensor-memory lane; velocity loops unrolled in chunks of eight (16
// columns), so velocity constants are compile-time operands.  Warp-collective
// (tcgen05.ld / st): every thread of the warp calls it; `store` selects the
// threads whose node is real.
template <class VSET>
__device__ __forceinline__ void collide_tmem(const CollideConst<float>& C, uint32_t tl, float Tw, float2* out,
                                             int NN, bool store) {
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    constexpr int NCH = (2 * Q + 15) / 16;
    // ---- moments: plain sums within a chunk, Kahan across chunks
    Acc<float> arho, aj0, aj1, aj2, ae;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        float v[16];
        tc_ld16(tl + 16 * c, v);
        float br = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f, be = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = 8 * c + j;
            if (i < Q) {
                const float f = v[2 * j], g = v[2 * j + 1];
                br += f;
                b0 += C.xi[i][0] * f;
                b1 += C.xi[i][1] * f;
                if (D == 3) b2 += C.xi[i][2] * f;
                be += C.s2[VSET::shell(i)] * f + g;
            }
        }
        arho.add(br);
        aj0.add(b0);
        aj1.add(b1);
        if (D == 3) aj2.add(b2);
        ae.add(be);
    }
    const float rho_d = arho.get();
    const float rho = 1.f + rho_d;
    const float inv_rho = 1.f / rho;
    const float u0 = aj0.get() * inv_rho, u1 = aj1.get() * inv_rho, u2 = D == 3 ? aj2.get() * inv_rho : 0.f;
    const float U = u0 * u0 + u1 * u1 + u2 * u2;
    float t = (ae.get() - rho * U - 2.f * C.cv * rho_d) * inv_rho / (2.f * C.cv);
    // P1 of velocity i at temperature offset tt; i is a constant after the
    // unrolling, so the shell coefficients of one shell are shared
    auto p1 = [&](int i, float tt, float& cd) {
        const int sh = VSET::shell(i);
        float c = C.xi[i][0] * u0 + C.xi[i][1] * u1;
        if (D == 3) c += C.xi[i][2] * u2;
        cd = c;
        const float k2 = 0.5f - 0.25f * U + 0.25f * tt * C.sC[sh];
        const float k1 = 1.0f - 0.5f * U + 0.5f * tt * C.sB[sh];
        const float k0 = -0.5f * U + 0.125f * U * U + 0.5f * tt * C.sA[sh] - 0.25f * tt * U * C.sB[sh] +
                         0.125f * tt * tt * C.sE[sh];
        return eq_poly1(c, k0, k1, k2);
    };
    // ---- isothermal wall correction (Eq. thermalBC), on the warps that hold such a node
    const bool iso = !(Tw != Tw);
    if (__any_sync(0xffffffffu, iso)) {
        const float tw = iso ? Tw - 1.f : t;
        const float rT0 = rho * (1.f + t), rT1 = rho * (1.f + tw);
#pragma unroll 1
        for (int c = 0; c < NCH; ++c) {
            float v[16];
            tc_ld16(tl + 16 * c, v);
            // runtime chunk, compile-time lane of the chunk: the shell
            // constants come from the per-velocity tables
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int i = 8 * c + j;
                if (i < Q) {
                    float cv = C.xi[i][0] * u0 + C.xi[i][1] * u1;
                    if (D == 3) cv += C.xi[i][2] * u2;
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
    float q0 = 0.f, q1 = 0.f, q2 = 0.f;
    const bool second = C.quasi || C.forced;
    // Kupershtokh exact-difference forcing (Sec. 4.3), du = F dt / rho: the
    // equilibrium at the shifted velocity v = u + du minus the one at u (the
    // relaxation's own P1), added in the relaxation pass
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, V = 0.f;
    if (C.forced) {
        v0 = u0 + C.force_dt[0] * inv_rho;
        v1 = u1 + C.force_dt[1] * inv_rho;
        v2 = D == 3 ? u2 + C.force_dt[2] * inv_rho : 0.f;
        V = v0 * v0 + v1 * v1 + v2 * v2;
    }
    // ---- relaxation (BGK); heat flux of the quasi-equilibrium term; forcing
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        float v[16];
        tc_ld16(tl + 16 * c, v);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = 8 * c + j;
            if (i < Q) {
                float cd;
                const float P1 = p1(i, t, cd);
                const float fe = C.w[i] * (rho * P1 + rho_d);
                const float ge = C.wg[i] * (rhoT * P1 + rhoT_d);
                const float f = v[2 * j], g = v[2 * j + 1];
                const float fn = f - fe, gn = g - ge;
                const float h = (C.s2[VSET::shell(i)] - 2.f * cd + U) * fn + gn;
                q0 += (C.xi[i][0] - u0) * h;
                q1 += (C.xi[i][1] - u1) * h;
                if (D == 3) q2 += (C.xi[i][2] - u2) * h;
                v[2 * j] = f - om * fn;
                v[2 * j + 1] = g - om * gn;
                if (C.forced) {
                    const int sh = VSET::shell(i);
                    float cw = C.xi[i][0] * v0 + C.xi[i][1] * v1;
                    if (D == 3) cw += C.xi[i][2] * v2;
                    const float k2 = 0.5f - 0.25f * V + 0.25f * t * C.sC[sh];
                    const float k1 = 1.0f - 0.5f * V + 0.5f * t * C.sB[sh];
                    const float k0 = -0.5f * V + 0.125f * V * V + 0.5f * t * C.sA[sh] - 0.25f * t * V * C.sB[sh] +
                                     0.125f * t * t * C.sE[sh];
                    v[2 * j] += C.w[i] * rho * (eq_poly1(cw, k0, k1, k2) - P1);
                }
                if (!second && store) out[i * NN] = make_float2(v[2 * j], v[2 * j + 1]);
            }
        }
        if (second) tm_st16(tl + 16 * c, v);
    }
    if (!second) return;
    tm_wait_st();
    const float a = om - om_pr;
    q0 *= C.quasi ? a : 0.f;
    q1 *= C.quasi ? a : 0.f;
    q2 *= C.quasi ? a : 0.f;
    // ---- the heat-flux correction of g
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        float v[16];
        tc_ld16(tl + 16 * c, v);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = 8 * c + j;
            if (i < Q) {
                float dq = C.xi[i][0] * q0 + C.xi[i][1] * q1;
                if (D == 3) dq += C.xi[i][2] * q2;
                if (store) out[i * NN] = make_float2(v[2 * j], v[2 * j + 1] + C.w[i] * dq);
            }
        }
    }
}

// ------------------------------------------------------------ the kernel
// NX x TY x TZ consumer threads (one arrival node each) and two producer warps.
// TC: the (y, z) contraction of each velocity as tensor-core products
// (128-node rows): D_f, D_g [128 x-nodes x 16] = A_f, A_g [x-nodes x kp
// source rows] . W [kp x 16 tile rows, zero padded], A split by the
// consumers and W by the host into TF32 hi and lo parts, three products
// (hi hi, hi lo, lo hi) into FP32 accumulators in tensor-memory columns
// 384 .. 415 (the node state uses 0 .. 383).
template <int VS, int NX, int TY, int TZ, bool TC>
__global__ void __launch_bounds__(NX * TY * TZ + 64, 1)
    k_step_rows_tmem(const float2* __restrict__ fg, float2* __restrict__ fgo, const float* __restrict__ bop,
                     const int32_t* __restrict__ head,
                     const TmRec* __restrict__ recs, const uint64_t* __restrict__ xmask,
                     const float* __restrict__ twt, const StepGeom G,
                     const CollideConst<float> C, const TmGeom T, int* __restrict__ status) {
    using VSET = VelSet<VS>;
    constexpr int Q = VSET::Q;
    constexpr int D = VSET::D;
    constexpr int NR = TY * TZ;                   // rows per tile
    constexpr int NT = NX * NR;                   // consumer threads
    constexpr int NW = NT / 32;                   // consumer warps
    constexpr int NPW = 2;                        // producer warps
    constexpr int XBW = NX + 4;                   // halo row of the x exchange
    constexpr int REC_BYTES = NR * 2 * int(sizeof(TmRec));
    static_assert(NT % 128 == 0 && NW <= 16 && 2 * Q <= TM_COLS, "tile shape");
    static_assert(NX % 32 == 0 && NX >= 32, "whole warps per row");
    static_assert(NX == 32 || NR <= 14, "named barriers 1 .. NR (one per row of more than one warp), 15");
    static_assert(!TC || (NX == 128 && NR <= 16 && NW * TM_COLS / 4 + 32 <= TM_ALLOC), "tensor-core variant");
    constexpr int B_FLOATS = 2 * 16;              // per K column of the weight operands (hi, lo) x 16 rows
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    unsigned char* stages = dyn_smem;                                         // [nst][rows | records]
    float2* XB = reinterpret_cast<float2*>(stages + size_t(T.nst) * T.stage_bytes);   // [2][NR][XBW]
    uint64_t* bars = reinterpret_cast<uint64_t*>(XB + 2 * NR * XBW);
    // full[nst], empty[nst], and one barrier that nothing completes (waited
    // on only under a test wait limit, so that the timeout path runs)
    uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2 * T.nst + 1);       // TMEM base, abort flag
    volatile int* abort_flag = reinterpret_cast<volatile int*>(slot + 1);
    // tensor-core variant: the A operands (f hi, f lo, g hi, g lo; 1024-byte
    // aligned) and the products' barrier
    const size_t a_off = ((reinterpret_cast<unsigned char*>(slot) + 16 - dyn_smem) + 1023) / 1024 * 1024;
    const uint32_t aop = smem_u32(dyn_smem + a_off);
    const uint32_t AOPB = uint32_t(NX * T.kp * 4);                            // bytes of one A operand
    const uint32_t mma_bar = aop + 4 * AOPB;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8u * uint32_t(T.nst);
    const uint32_t st0 = smem_u32(stages);
    const int NN = int(G.n_nodes);
    const int N1 = G.N[1], N2 = D == 3 ? G.N[2] : 1;
    const bool py = G.periodic[1] != 0;
    const long long lim = wait_limit(status);
    if (tid == 0) {
        for (int s = 0; s < T.nst; ++s) {
            mbar_init(full0 + 8u * uint32_t(s), 1);
            mbar_init(empty0 + 8u * uint32_t(s), NW);
        }
        mbar_init(full0 + 16u * uint32_t(T.nst), 1);
        if (TC) mbar_init(mma_bar, 1);
        *abort_flag = 0;
    }
    if (warp == 0) {
        tc_alloc(smem_u32(slot), TM_ALLOC);
        tc_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(slot);

    if (warp >= NW) {
        // ------------------------------------------------ producer warps
        // The velocities of this CTA's tiles as one sequence k = (tile, i);
        // producer warp pw issues k = pw, pw + NPW, ... into stages
        // k mod nst (nst is a multiple of NPW).  The copy list of its next
        // velocity is loaded while the current one is issued, so its L2
        // latency stays off the issue path.
        const int pw = warp - NW;
        int s = pw, ph = 0;              // stage, and the parity of its next use
        long long seq = 0;               // velocities issued by this warp
        const int my_tiles = int(blockIdx.x) < T.ntiles ? (T.ntiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
        const int total = my_tiles * Q;
        int cur_tile = -1, y0 = 0, z0 = 0, tc = 0;
        struct Hd {
            int n, rows, e, sl;          // runs, rows; this lane's run and its first slot
        };
        auto fetch = [&](int k) {
            Hd hd{0, 0, 0, 0};
            if (k < total) {
                const int tile = int(blockIdx.x) + (k / Q) * int(gridDim.x), i = k % Q;
                const int tcl = py ? 0 : tile % T.ntile_y;
                const int32_t* h = head + (size_t(i) * T.n_tc + tcl) * TM_HEAD;
                hd.n = __ldg(h);
                hd.rows = __ldg(h + 1);
                hd.e = __ldg(h + 2 + lane);
                hd.sl = __ldg(h + 2 + TM_MAX_RUNS + lane);
            }
            return hd;
        };
        Hd ha = fetch(pw);
#pragma unroll 1
        for (int k = pw; k < total; k += NPW) {
            const Hd hb = fetch(k + NPW);
            const int kt = k / Q, i = k - kt * Q;
            if (kt != cur_tile) {
                cur_tile = kt;
                const int tile = int(blockIdx.x) + kt * int(gridDim.x);
                const int ty = tile % T.ntile_y, tz = tile / T.ntile_y;
                y0 = ty * TY;
                z0 = tz * TZ;
                tc = py ? 0 : ty;
            }
            if (seq * NPW + pw >= T.nst) {
                // the stage's previous contents have been read by every consumer warp
                bool ok = !*abort_flag && mbar_wait(empty0 + 8u * uint32_t(s), uint32_t(ph ^ 1), lim);
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
            const uint32_t fb = full0 + 8u * uint32_t(s);
            const uint32_t sb = st0 + uint32_t(s) * uint32_t(T.stage_bytes);
            const uint32_t b_bytes = TC ? uint32_t(B_FLOATS * T.kp * 4) : 0u;
            if (lane == 0) mbar_arrive_expect_tx(fb, uint32_t(ha.rows * NX * 8 + REC_BYTES) + b_bytes);
            __syncwarp();
            if (lane < ha.n) {
                // this lane's run: population, first y and z (relative to the tile), rows
                const int e = ha.e;
                const int src = e & 63, len = (e >> 22) & 63;
                int ya = y0 + ((e >> 6) & 255) - 128;
                int z = D == 3 ? z0 + ((e >> 14) & 255) - 128 : 0;
                if (D == 3) {
                    z += z < 0 ? N2 : 0;
                    z -= z >= N2 ? N2 : 0;
                }
                z = SLLBM_CHK(z, N2, G.status, SLLBM_DEV_BAD_NODE);
                z = min(max(z, 0), N2 - 1);              // every copy stays inside the mesh
                const float2* pop = fg + size_t(SLLBM_CHK(src, Q, G.status, SLLBM_DEV_BAD_POP)) * NN +
                                    size_t(z) * N1 * NX;
                const uint32_t dst = sb + uint32_t(ha.sl * NX * 8);
                if (py) {
                    // periodic y: a run that crosses the last row continues at row 0
                    ya += ya < 0 ? N1 : 0;
                    ya -= ya >= N1 ? N1 : 0;
                    ya = min(max(ya, 0), N1 - 1);
                    const int l1 = min(len, N1 - ya);
                    bulk_g2s(dst, pop + size_t(ya) * NX, uint32_t(l1 * NX * 8), fb);
                    if (len > l1) bulk_g2s(dst + uint32_t(l1 * NX * 8), pop, uint32_t((len - l1) * NX * 8), fb);
                } else {
                    ya = SLLBM_CHK(ya, N1, G.status, SLLBM_DEV_BAD_NODE);
                    ya = min(max(ya, 0), N1 - len);      // every copy stays inside the mesh
                    bulk_g2s(dst, pop + size_t(ya) * NX, uint32_t(len * NX * 8), fb);
                }
            }
            if (lane == 31)
                bulk_g2s(sb + uint32_t(T.rows_bytes), recs + (size_t(i) * T.n_tc + tc) * (NR * 2),
                         uint32_t(REC_BYTES), fb);
            if (TC && lane == 30)
                bulk_g2s(sb + uint32_t(T.rows_bytes + REC_BYTES), bop + (size_t(i) * T.n_tc + tc) * B_FLOATS * T.kp,
                         b_bytes, fb);
            ++seq;
            s += NPW;
            if (s >= T.nst) {
                s -= T.nst;
                ph ^= 1;
            }
            ha = hb;
        }
        // on an abort: wait (bounded, default limit) for every copy issued,
        // so that none lands in shared memory after the CTA has exited
        if (*abort_flag && lane == 0) {
            // this warp's last nst / NPW velocities: global sequence numbers
            // pw + NPW q for its q-th velocity
            const long long per = T.nst / NPW;
            const long long first = seq > per ? seq - per : 0;
            for (long long q = first; q < seq; ++q) {
                const long long g = pw + NPW * q;
                mbar_wait(full0 + 8u * uint32_t(g % T.nst), uint32_t((g / T.nst) & 1));
            }
        }
    } else {
        // ------------------------------------------------ consumers
        const int x = tid % NX, r = tid / NX;
        const int ry = r % TY, rz = r / TY;
        const uint32_t tl = tbase + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(TM_COLS * (warp >> 2));
        int s = 0, ph = 0, xb = 0, mph = 0;
        for (int tile = blockIdx.x; tile < T.ntiles; tile += gridDim.x) {
            const int ty = tile % T.ntile_y, tz = tile / T.ntile_y;
            const int y = ty * TY + ry, z = D == 3 ? tz * TZ + rz : 0;
            const bool real = y < N1;
            const int n = x + NX * (y + N1 * z);
            // velocities whose x factor needs the row exchange, for this tile
            // class: read from global memory, so that every thread of a row
            // takes the same barriers whatever the stage holds
            const uint64_t xm = __ldg(xmask + (py ? 0 : ty));
#pragma unroll 1
            for (int i = 0; i < Q; ++i) {
                const uint32_t fb = full0 + 8u * uint32_t(s);
                // under a test wait limit the first velocity also waits on the
                // barrier that nothing completes, so that the wait runs out
                // whatever the timing (sllbm_debug_wait_limit)
                bool live = !*abort_flag;
                if (live && (!mbar_wait(fb, uint32_t(ph), lim) ||
                             (lim < kWaitLimit && i == 0 && !mbar_wait(full0 + 16u * uint32_t(T.nst), 0, lim)))) {
                    atomicOr(status, SLLBM_DEV_COPY_TIMEOUT);
                    *abort_flag = 1;
                    live = false;
                }
                // after an abort the stage may never have been written: read
                // no offsets from it (an empty equilibrium record instead)
                const unsigned char* st = stages + size_t(s) * T.stage_bytes;
                const TmRec* rp = reinterpret_cast<const TmRec*>(st + T.rows_bytes) + (r * 2 + (x & 1));
                const int4 q0 = reinterpret_cast<const int4*>(rp)[0];
                const int4 q1 = reinterpret_cast<const int4*>(rp)[1];
                const int meta = live ? q0.x : int(REC_EQ), ntap = live ? q0.y : 0;
                const int dx0 = min(max(q0.z, -2), 0);
                const float wx0 = __int_as_float(q0.w), wx1 = __int_as_float(q1.x), wx2 = __int_as_float(q1.y);
                const unsigned char* bx = st + 8 * x;
                float2 sum = make_float2(0.f, 0.f);
                if (!TC && ntap > 0) {
                    const int4 q2 = reinterpret_cast<const int4*>(rp)[2];
                    const int4 q3 = reinterpret_cast<const int4*>(rp)[3];
                    const int4 q4 = reinterpret_cast<const int4*>(rp)[4];
                    const int4 q5 = reinterpret_cast<const int4*>(rp)[5];
                    const int off[9] = {q1.z, q1.w, q2.x, q2.y, q2.z, q2.w, q3.x, q3.y, q3.z};
                    const float w[9] = {__int_as_float(q3.w), __int_as_float(q4.x), __int_as_float(q4.y),
                                        __int_as_float(q4.z), __int_as_float(q4.w), __int_as_float(q5.x),
                                        __int_as_float(q5.y), __int_as_float(q5.z), __int_as_float(q5.w)};
                    // two accumulators (even and odd taps): half the dependent chain
                    float2 sum1 = make_float2(0.f, 0.f);
                    auto tap = [&](int k) {
                        const float2 v = *reinterpret_cast<const float2*>(
                            bx + SLLBM_CHK(off[k], T.rows_bytes, G.status, SLLBM_DEV_BAD_SMEM));
                        if (k & 1) sum1 = __ffma2_rn(make_float2(w[k], w[k]), v, sum1);
                        else sum = __ffma2_rn(make_float2(w[k], w[k]), v, sum);
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
                    sum = __fadd2_rn(sum, sum1);
                }
                if constexpr (TC) {
                    // split the staged rows into TF32 hi and lo parts, K-major
                    // (thread (x, r) takes the source rows k = r, r + NR, ..);
                    // rows beyond the velocity's own are zero
                    const int kp = T.kp;
                    const int rows = live ? __ldg(head + (size_t(i) * T.n_tc + (py ? 0 : ty)) * TM_HEAD + 1) : 0;
                    const uint32_t sa = smem_u32(st);
                    for (int k = r; k < kp; k += NR) {
                        float2 v = make_float2(0.f, 0.f);
                        if (k < rows) v = lds2_tm(sa + uint32_t(k * NX * 8 + 8 * x));
                        const float fh = to_tf32(v.x), gh = to_tf32(v.y);
                        const uint32_t o = aop + tf32_canon(x, k, kp);
                        sts1(o, fh);
                        sts1(o + AOPB, to_tf32(v.x - fh));
                        sts1(o + 2 * AOPB, gh);
                        sts1(o + 3 * AOPB, to_tf32(v.y - gh));
                    }
                    fence_async_smem();       // generic-proxy writes -> the tensor cores
                    tc_fence_before();
                    row_bar(15, NT);          // every consumer has written its part
                    if (tid == 0) {
                        tc_fence_after();
                        constexpr uint32_t id = tc_idesc_tf32(128, 16);
                        const uint32_t bb = sa + uint32_t(T.rows_bytes + REC_BYTES);   // W hi | W lo
                        const uint32_t sbo = uint32_t(kp * 32);
#pragma unroll 1
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t d = tbase + 384u + 16u * uint32_t(h);
                            const uint32_t ahi = aop + 2u * uint32_t(h) * AOPB, alo = ahi + AOPB;
#pragma unroll 1
                            for (int kk = 0; kk < kp / 8; ++kk) {
                                const uint64_t bh = tc_sdesc(bb + 256u * kk, 128, sbo);
                                const uint64_t bl = tc_sdesc(bb + uint32_t(16 * kp * 4) + 256u * kk, 128, sbo);
                                const uint64_t ah = tc_sdesc(ahi + 256u * kk, 128, sbo);
                                const uint64_t al = tc_sdesc(alo + 256u * kk, 128, sbo);
                                tc_mma_tf32(d, ah, bh, id, kk > 0 ? 1u : 0u);
                                tc_mma_tf32(d, ah, bl, id, 1u);
                                tc_mma_tf32(d, al, bh, id, 1u);
                            }
                        }
                        tc_commit(mma_bar);
                    }
                    // the products are complete (a wait that runs out waits
                    // once more with the default bound, so that no product
                    // is in flight when its operands or accumulators are reused)
                    if (!mbar_wait(mma_bar, uint32_t(mph), lim)) {
                        mbar_wait(mma_bar, uint32_t(mph));
                        atomicOr(status, SLLBM_DEV_TC_TIMEOUT);
                        *abort_flag = 1;
                    }
                    mph ^= 1;
                    tc_fence_after();
                    const uint32_t td = tbase + (uint32_t(32 * (warp & 3)) << 16) + 384u + uint32_t(r);
                    sum.x = tm_ld1(td);
                    sum.y = tm_ld1(td + 16u);
                    tc_fence_before();
                }
                // this warp has read the stage: release it to the producer
                __syncwarp();
                if (lane == 0) mbar_arrive(empty0 + 8u * uint32_t(s));
                float2 o = sum;
                if ((xm >> i) & 1) {
                    // x factor: the three x taps of the row sums, through a
                    // halo row (periodic images of the first and last two)
                    float2* xr = XB + (xb * NR + r) * XBW;
                    xr[x + 2] = sum;
                    if (x < 2) xr[x + NX + 2] = sum;
                    if (x >= NX - 2) xr[x - NX + 2] = sum;
                    if (NX == 32) __syncwarp();       // a row of one warp
                    else row_bar(1 + r, NX);
                    const float2* t3 = xr + x + 2 + dx0;   // dx0 in [-2, 0]: indices x .. x + 4
                    o = __fmul2_rn(make_float2(wx0, wx0), t3[0]);
                    o = __ffma2_rn(make_float2(wx1, wx1), t3[1], o);
                    o = __ffma2_rn(make_float2(wx2, wx2), t3[2], o);
                    xb ^= 1;
                }
                const int kind = meta & 15;
                const int bid = (meta >> 4) & 15;
                if (kind == REC_EQ) {
                    o.x = C.eqf[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                    o.y = C.eqg[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                } else if (kind == REC_BB || kind == REC_BB_ISO) {
                    o.x += C.mw[SLLBM_CHK(bid, 2, G.status, SLLBM_DEV_BAD_REC)][i];
                }
                tm_st2(tl + 2 * i, o.x, o.y);
                if (++s == T.nst) {
                    s = 0;
                    ph ^= 1;
                }
            }
            tm_wait_st();
            const int cls = (x & 1) + G.ncls[0] * ((py ? (y & 1) : (real ? y : 0)) + G.ncls[1] * (D == 3 ? (z & 1) : 0));
            const float Tw = real ? __ldg(twt + cls) : __int_as_float(0x7fc00000);
            collide_tmem<VSET>(C, tl, Tw, fgo + n, NN, real && !*abort_flag);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tbase, TM_ALLOC);
    }
}

size_t rows_tmem_smem_bytes(int D, int nx, const TmGeom& T);

template <int VS, int NX, int TY, int TZ, bool TC>
int launch_step_rows_tmem(const float2* fg, float2* fgo, const float* bop, const int32_t* head, const TmRec* recs,
                          const uint64_t* xmask, const float* tw, const StepGeom& G, const CollideConst<float>& C,
                          const TmGeom& T, int* status, cudaStream_t stream, int grid) {
    constexpr int NR = TY * TZ;
    const size_t smem = rows_tmem_smem_bytes(VelSet<VS>::D, NX, T);
    if (cudaFuncSetAttribute(k_step_rows_tmem<VS, NX, TY, TZ, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem)) != cudaSuccess)
        return SLLBM_ERR_CUDA;
    k_step_rows_tmem<VS, NX, TY, TZ, TC><<<grid, NX * NR + 64, smem, stream>>>(fg, fgo, bop, head, recs, xmask, tw, G, C, T,
                                                                               status);
    return cudaGetLastError() == cudaSuccess ? SLLBM_OK : SLLBM_ERR_CUDA;
}

}  // namespace sllbm
