/*
 * sllbm.h -- C ABI of the GB300 semi-Lagrangian lattice Boltzmann library.
 *
 * The library implements the fused per-node pull step of the compressible
 * semi-Lagrangian lattice Boltzmann method (SLLBM) of Spelten, Wilde,
 * Bedrunka, Reith and Foysi (arXiv 2412.09051):
 *   - stream by interpolation at the departure point (Sec. 3.1, Eq. 1 and
 *     Eq. intf: order-p Lagrange interpolation in the departure cell),
 *   - density / momentum / energy moments (Sec. 3.1, moment equations),
 *   - relaxation towards the order-4 Hermite equilibrium with the
 *     quasi-equilibrium term for Pr != 1 (Sec. 3.1, Eq. 1),
 *   - the boundary schemes of Sec. 3.3: equilibrium (3.3.1), bounce-back and
 *     isothermal wall (3.3.2, Eq. thermalBC) and zero-gradient outlet (3.3.3),
 * on one CUDA device (sm_103a).  A one-time FP64 setup pass traces every
 * departure point, inverts curved cell maps by Newton iteration and stores
 * departure records (Sec. 3.1: departure point x_AP - dt zeta_i).
 *
 * Conventions
 *   - Every call returns an int status: SLLBM_OK (0) or a negative SLLBM_ERR_*.
 *     No C++ exception crosses this boundary.  sllbm_last_error() returns a
 *     human-readable message for the last failing call on a context.
 *   - Units: gas constant R = 1, lattice reference state rho0 = T0 = 1,
 *     c_v = 1/(gamma - 1); abscissae zeta_i = xi_i (sqrt(T0) = 1).
 *   - Node numbering is structured: n = k0 + N0 (k1 + N1 k2), first dimension
 *     fastest; periodic duplicates are removed.  Cell numbering likewise.
 *   - Population arrays are [Q][N] (velocity-major, node fastest).
 *   - Pointers flagged `on_device` are CUDA device pointers on the context's
 *     device; otherwise host pointers (pageable or pinned).  The caller owns
 *     every buffer it passes; the context owns only what it allocates itself
 *     and frees it in sllbm_destroy().
 *   - All work is enqueued on the context's stream.  Calls that return data
 *     to host memory synchronise that stream before returning.
 *   - There is no CPU fallback: a context can only be created on a device of
 *     compute capability 10.3 (sm_103a); otherwise SLLBM_ERR_ARCH.
 */
#ifndef SLLBM_H
#define SLLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define SLLBM_OK                 0
#define SLLBM_ERR_ARG           -1   /* invalid argument or descriptor          */
#define SLLBM_ERR_CUDA          -2   /* a CUDA runtime call failed               */
#define SLLBM_ERR_ARCH          -3   /* device is not sm_103 or not present      */
#define SLLBM_ERR_NOMEM         -4   /* device allocation failed                 */
#define SLLBM_ERR_DP_NOT_FOUND  -5   /* setup: a departure point was not located
                                        within the Newton / cell-walk caps       */
#define SLLBM_ERR_UNSTABLE      -6   /* non-positive density or temperature      */
#define SLLBM_ERR_STATE         -7   /* call out of order (e.g. step before init) */
#define SLLBM_ERR_UNSUPPORTED   -8   /* combination not built in this library    */

/* ------------------------------------------------------------------ enums */
/* Mesh kinds (Sec. 3.1: cells with order-p Lagrange support points at the
 * Gauss-Lobatto-Chebyshev positions -cos(pi k / p), Tab. 2 caption). */
#define SLLBM_MESH_BOX       0  /* periodic in every dimension, uniform cells on [0, L_d)    */
#define SLLBM_MESH_CHANNEL   1  /* x,z periodic uniform; y in [0, L_y] with tanh clustering:
                                   y_j = L_y/2 [1 - tanh(s (1 - 2 j / C_y)) / tanh(s)]        */
#define SLLBM_MESH_MIXING    2  /* x,z periodic uniform; y in [-L_y/2, L_y/2]: `central`
                                   uniform cells, neighbours grow by the factor s outwards   */
#define SLLBM_MESH_NACA      3  /* 2D O-grid around a NACA-00tt profile (closed trailing edge
                                   form of the thickness formula); surface point at angle
                                   phi = 2 pi s / C_0: x = 1 - (1 - cos phi)/2
                                   - 0.25 |sin phi| (1 + cos phi)/2, y = sign(sin phi) y_t(x);
                                   radial line to the far-field point at the same angle;
                                   dim 0 around (periodic),
                                   dim 1 radial, growth factor s per cell up to a circle of
                                   radius L_1 about mid-chord; isoparametric degree-p cells  */
#define SLLBM_MESH_EXPLICIT  4  /* axis-aligned cells on the caller's vertex coordinates per
                                   dimension (vertices[d]: cells[d] + 1 strictly increasing
                                   values, lengths taken from them); x and z periodic, y
                                   periodic when both boundary kinds are SLLBM_BC_PERIODIC,
                                   else bounded by them; a periodic dimension starts at 0.
                                   Uniform periodic dimensions keep every streaming mode;
                                   non-uniform ones take the gather streaming               */

/* Velocity sets (Sec. 3.2).  Ordering: index 0 rest, then shells; inside a
 * shell of n points the second half are the negatives of the first half.
 *   D2Q9   classic lattice, xi in {0, +-sqrt3}^2 (classic-LBM special case, Sec. 2)
 *   D2Q19  degree-9 cubature: rest, ring r^2 = (48 - 8 sqrt15)/7 at k 60 deg,
 *          ring r = 2 sqrt2 at 30 + k 60 deg, ring r^2 = (48 + 8 sqrt15)/7 at k 60 deg
 *   D2Q25  product 5-point Gauss-Hermite rule (degree 9), x fastest over
 *          nodes {0, r1, r2, -r1, -r2}, r1,2 = sqrt(5 -+ sqrt10)
 *   D3Q45  degree-9 cubature: rest, icosahedron (cyclic perms of (0,+-phi,+-1)) at
 *          radius sqrt3, dodecahedron ((+-1)^3, cyclic perms of (0,+-1/phi,+-phi)) at
 *          radius 3, icosahedron (same orientation) at radius sqrt15 */
#define SLLBM_D2Q9    0
#define SLLBM_D2Q19   1
#define SLLBM_D2Q25   2
#define SLLBM_D3Q45   3
/* Sets run by the generic kernels (the velocity count known at run time, the
 * per-velocity constants in a device table; gather streaming, no learned
 * collision), created with sllbm_create_desc:
 *   D3Q125  product 5-point Gauss-Hermite rule (degree 9), x fastest over the
 *           nodes of D2Q25
 *   CUSTOM  the caller's abscissae xi[Q][D] and weights w[Q] (Q <= SLLBM_QMAX_GENERIC,
 *           in units of sqrt(T0)): the set must be symmetric under xi -> -xi and
 *           reproduce the weight function's moments to second order (sum w = 1,
 *           sum w xi = 0, sum w xi xi = identity, to 1e-10); the equilibrium
 *           of Sec. 3.1 is exact only where the set integrates degree 9 */
#define SLLBM_D3Q125        4
#define SLLBM_VELSET_CUSTOM 5
#define SLLBM_QMAX_GENERIC  128

typedef struct {
    int32_t kind;          /* SLLBM_D2Q9 .. SLLBM_VELSET_CUSTOM                          */
    int32_t Q;             /* CUSTOM: number of velocities (else ignored)              */
    int32_t D;             /* CUSTOM: dimension, equal to the mesh's (else ignored)    */
    int32_t reserved;      /* 0                                                        */
    const double* xi;      /* CUSTOM: host array xi[Q][D]; read during the call only   */
    const double* w;       /* CUSTOM: host array w[Q]; read during the call only       */
} sllbm_velset_desc;

/* Boundary kinds (Sec. 3.3).  Boundary id 0 is the low-y side of channel /
 * mixing meshes and the profile wall of the NACA O-grid; id 1 is the high-y
 * side and the O-grid far field. */
#define SLLBM_BC_PERIODIC     0
#define SLLBM_BC_EQUILIBRIUM  1  /* f_i(AP) = f_i^eq(rho_w, u_w, T_w)                      (3.3.1) */
#define SLLBM_BC_BOUNCEBACK   2  /* f_i(AP) = f_ibar(x_W + iota) [+ 2 w_i rho_w zeta_i.u_w] (3.3.2) */
#define SLLBM_BC_ISOTHERMAL   3  /* bounce-back plus f += f^eq(T_w) - f^eq(T)    (Eq. thermalBC) */
#define SLLBM_BC_OUTLET       4  /* f_i(AP) = f_i(x_AP + zeta_i dt)                        (3.3.3) */
#define SLLBM_BC_FARFIELD     5  /* equilibrium where the wall point lies upstream of mid-chord,
                                    outlet downstream (NACA far field)                           */

#define SLLBM_FP64  0   /* populations and arithmetic in FP64                       */
#define SLLBM_FP32  1   /* populations stored in FP32 as deviations from w_i rho0 (f)
                           and w_i rho0 T0 (2 c_v - D) (g); compensated FP32 moments  */

#define SLLBM_STREAM_AUTO        0  /* structured kernel where cells are axis-aligned, else gather */
#define SLLBM_STREAM_GATHER      1  /* one departure record per (node, velocity), node state in
                                       registers                                                 */
#define SLLBM_STREAM_STRUCTURED  2  /* one record per (velocity, translation class of nodes); the
                                       warp-tiled kernel with the node state in shared memory
                                       where eligible (p = 2 or 4, periodic x (and z in 3D), x
                                       taps within +-p nodes), else one thread per node          */
#define SLLBM_STREAM_STRUCTURED_NODE 3  /* class records, always one thread per node              */
#define SLLBM_STREAM_TILED_REG   4  /* warp-tiled kernel with the node state in registers (the
                                       kernel that carries the learned collision); p = 2 only,
                                       p = 4 runs the order-4 shared-memory warp-tiled kernel    */
#define SLLBM_STREAM_GATHER_SMEM 5  /* per-record gather with the node state in shared memory    */
#define SLLBM_STREAM_ROW_COPY    6  /* as SLLBM_STREAM_STRUCTURED, but where one block takes a
                                       periodic row (FP32, p = 2, D2Q19 rows of 32..256 nodes,
                                       D3Q45 rows of 32..128) the source rows of each velocity are
                                       staged in shared memory by the bulk-copy (TMA) engine, six
                                       velocities ahead, instead of loaded by every thread; other
                                       meshes run the SLLBM_STREAM_STRUCTURED kernels             */
#define SLLBM_STREAM_ROWS_TMEM   7  /* as SLLBM_STREAM_STRUCTURED, but where the mesh allows it
                                       (FP32, p = 2, D3Q45 rows of 32, 64 or 128 nodes or D2Q19
                                       rows of 32..256, periodic x and z, x taps within two
                                       nodes) a persistent kernel takes tiles of 512 nodes (whole
                                       x rows), keeps each node's 2Q streamed values in tensor
                                       memory and stages every source row a tile reads once in
                                       shared memory with the bulk-copy (TMA) engine.  With
                                       D3Q45, SLLBM_STREAM_AUTO and SLLBM_STREAM_STRUCTURED use
                                       this kernel where SLLBM_STREAM_ROWS_PAIRS does not apply
                                       (rows of 32 nodes)                                        */
#define SLLBM_STREAM_ROW_SMEM    8  /* as SLLBM_STREAM_STRUCTURED without the tensor-memory
                                       row-tile kernel (the one-block-per-row and warp-tiled
                                       kernels): for comparisons                                 */
#define SLLBM_STREAM_TENSOR      9  /* the SLLBM_STREAM_ROWS_TMEM kernel with the (y, z) part of
                                       the streaming on the tensor cores: per velocity and tile
                                       the product of the staged source rows (128 x-nodes x the
                                       velocity's rows, f and g separately) with the tile's
                                       interpolation weights (its rows x 4 tile rows), tcgen05
                                       kind::tf32 with both operands split into TF32 hi and lo
                                       parts (hi hi + hi lo + lo hi: FP32 accuracy), FP32
                                       accumulators in tensor memory; D3Q45 rows of 128 nodes only
                                       (elsewhere as SLLBM_STREAM_ROWS_TMEM), opt-in: slower than
                                       the CUDA-core contraction                                 */
#define SLLBM_STREAM_ROWS_PAIRS 10  /* the SLLBM_STREAM_ROWS_TMEM design with two arrival nodes
                                       (x even, x + 1) per consumer thread while streaming, one
                                       TMA tensor copy per (source population, velocity, tile) and
                                       stages of up to six velocities: D3Q45 rows of 64 or 128
                                       nodes (orders 2 and 4; tiles of 256 nodes, two CTAs per
                                       SM, opposite velocities collided in pairs), D2Q19 rows of
                                       64 or 128 (tiles of 512 nodes, one CTA per SM), periodic x
                                       and z (elsewhere as SLLBM_STREAM_ROWS_TMEM).  With D3Q45,
                                       SLLBM_STREAM_AUTO and SLLBM_STREAM_STRUCTURED use this
                                       kernel wherever it applies                                */

/* ------------------------------------------------------------------ descriptors */
typedef struct {
    int32_t kind;          /* SLLBM_BC_* */
    double  rho;           /* wall / inflow density rho_w     */
    double  u[3];          /* wall / inflow velocity u_w      */
    double  T;             /* wall / inflow temperature T_w   */
} sllbm_bc;

typedef struct {
    int32_t  kind;         /* SLLBM_MESH_*                                         */
    int32_t  dim;          /* D = 2 or 3                                           */
    int32_t  p;            /* Lagrange order, 1..4                                 */
    int32_t  cells[3];     /* cells per dimension                                  */
    double   length[3];    /* domain extent per dimension (NACA: [chord=1, R, -])  */
    double   stretch;      /* tanh parameter (channel), growth factor (mixing, NACA) */
    int32_t  central;      /* mixing: number of uniform central cells in y         */
    double   thickness;    /* NACA relative thickness t (0.12 for NACA-0012)       */
    sllbm_bc bc[2];        /* boundary ids 0 and 1                                 */
    const double* vertices[3];  /* EXPLICIT: host arrays of cells[d] + 1 vertex
                                   coordinates per dimension, read during the call
                                   (other kinds: ignored)                              */
} sllbm_mesh_desc;

typedef struct {
    double  dt;            /* time step                                             */
    double  gamma;         /* ratio of specific heats                                */
    double  Pr;            /* Prandtl number                                          */
    double  mu_ref;        /* mu(T) = mu_ref (T / T_ref)^mu_exp  (Sec. 4.3 power law) */
    double  T_ref;
    double  mu_exp;
    int32_t precision;     /* SLLBM_FP64 / SLLBM_FP32                                */
    int32_t stream_mode;   /* SLLBM_STREAM_*                                          */
    int32_t device;        /* CUDA device ordinal                                      */
    int32_t max_newton;    /* setup Newton cap (0: default 40)                        */
    int32_t max_walk;      /* setup cell-walk cap (0: default 64)                     */
    void*   stream;        /* cudaStream_t to enqueue on (NULL: a stream owned by the ctx) */
} sllbm_params;

typedef struct {
    int64_t n_nodes;       /* N                                                  */
    int32_t Q, dim, p;
    int32_t nodes[3];      /* nodes per dimension                                */
    int32_t cells[3];
    int32_t precision;
    int32_t stream_mode;   /* resolved mode actually used                       */
    int64_t state_bytes;   /* device bytes of one population buffer pair (f and g) */
    int64_t table_bytes;   /* device bytes of the departure records used by step   */
    int64_t n_records;     /* number of departure records                          */
    int64_t n_boundary_records;  /* records whose trajectory left the domain       */
    int64_t n_isothermal_nodes;  /* nodes with an isothermal-wall trajectory       */
    char     step_kernel[32];     /* name of the kernel the last step launched
                                     ("" before the first step)                   */
} sllbm_info_t;

typedef struct sllbm_ctx sllbm_ctx;

/* ------------------------------------------------------------------ lifecycle */

/* Create a context: builds the mesh and the velocity set on the host (FP64),
 * runs the FP64 departure-point setup kernels on the device (Sec. 3.1: DP =
 * x_AP - dt zeta_i; curved cells inverted by Newton iteration; Sec. 3.3 for
 * trajectories that leave the domain) and allocates two population buffers.
 * Errors: SLLBM_ERR_ARG (bad descriptor), SLLBM_ERR_ARCH (not sm_103),
 * SLLBM_ERR_NOMEM, SLLBM_ERR_DP_NOT_FOUND (setup caps exceeded), SLLBM_ERR_CUDA.
 * On error *out is NULL and the message is available from sllbm_last_error(NULL). */
int sllbm_create(const sllbm_mesh_desc* mesh, int32_t velset, const sllbm_params* params,
                 sllbm_ctx** out);

/* sllbm_create with a velocity-set descriptor (Sec. 3.2): the four sets above
 * by kind (exactly as sllbm_create), D3Q125, or a caller's set.  The generic
 * kinds (D3Q125, CUSTOM) take the gather streaming whatever params->stream_mode
 * asks, orders p = 2, 3, 4, FP64 or FP32; the learned collision is not
 * available on them (SLLBM_ERR_UNSUPPORTED).
 * Errors as sllbm_create; a custom set that fails the checks above gives
 * SLLBM_ERR_ARG before any device work. */
int sllbm_create_desc(const sllbm_mesh_desc* mesh, const sllbm_velset_desc* velset, const sllbm_params* params,
                      sllbm_ctx** out);

/* Free everything the context owns.  NULL is accepted. */
int sllbm_destroy(sllbm_ctx* ctx);

/* Device memory from the caller (e.g. a framework's caching allocator).
 * Contexts created after this call take every device buffer they own (state
 * buffers, departure tables, scratch, the staging of host reads) from
 * alloc(bytes, user) and give it back with release(ptr, user), from the
 * thread that calls the library; contexts created before keep their own.
 * The memory must be device memory of the context's GPU and 256-byte
 * aligned: anything else is released at once and the call that asked for it
 * fails with SLLBM_ERR_ARG; alloc returning NULL fails it with
 * SLLBM_ERR_NOMEM.  A context releases its buffers in sllbm_destroy (after
 * synchronising its stream) and temporaries before the call that took them
 * returns.  Both NULL: cudaMalloc / cudaFree again (the default); exactly one
 * NULL: SLLBM_ERR_ARG.  Process-wide; not synchronised with concurrent
 * sllbm_create calls on other threads.  The training context
 * (sllbm_train_create) allocates with cudaMalloc. */
typedef void* (*sllbm_alloc_fn)(size_t bytes, void* user);
typedef void (*sllbm_free_fn)(void* ptr, void* user);
int sllbm_set_allocator(sllbm_alloc_fn alloc, sllbm_free_fn release, void* user);

/* Message of the last failing call on ctx (ctx may be NULL: last create error). */
const char* sllbm_last_error(const sllbm_ctx* ctx);

/* Sizes and resolved options of a context. */
int sllbm_info(const sllbm_ctx* ctx, sllbm_info_t* out);

/* Node coordinates, x[N][D] (row per node), FP64. */
int sllbm_node_coords(sllbm_ctx* ctx, double* x, int32_t on_device);

/* Velocity set: xi[Q][D], w[Q], opp[Q] (index of -xi_i).  Host pointers. */
int sllbm_velocity_set(const sllbm_ctx* ctx, double* xi, double* w, int32_t* opp);

/* ------------------------------------------------------------------ state */

/* Initialise the populations to the equilibria f^eq, g^eq (Sec. 3.1) of the
 * given macroscopic fields rho[N], u[N][D], T[N] (FP64). */
int sllbm_init_state(sllbm_ctx* ctx, const double* rho, const double* u, const double* T,
                     int32_t on_device);

/* Full populations f[Q][N], g[Q][N] in FP64 (storage deviations plus their
 * reference values). */
int sllbm_get_state(sllbm_ctx* ctx, double* f, double* g, int32_t on_device);
int sllbm_set_state(sllbm_ctx* ctx, const double* f, const double* g, int32_t on_device);

/* Native storage, bitwise checkpoint / restore of the current step's
 * populations: deviations from the reference values, FP32 or FP64 per the
 * context's precision, interleaved per population and node as (f, g) pairs:
 * element [i][n][0] = f_i(n) - w_i, [i][n][1] = g_i(n) - w_i (2 c_v - D).
 * Size 2 Q N elements. */
int sllbm_get_state_raw(sllbm_ctx* ctx, void* fg, int32_t on_device);
int sllbm_set_state_raw(sllbm_ctx* ctx, const void* fg, int32_t on_device);

/* Node layers of constant x index x0 .. x0 + nx - 1 (every (y, z) row, every
 * population) of the current state, copied to / from the caller's buffer in
 * the raw format of sllbm_get_state_raw restricted to those x: element
 * [i][row][k][0] = f_i - w_i and [i][row][k][1] = g_i - w_i (2 c_v - D) at
 * x = x0 + k, row = y + N_y z; 2 Q N_y N_z nx values of the context's
 * precision.  This is the halo exchange of a domain decomposition along x
 * (the paper's runs are multi-node, Sec. 4; it does not describe the
 * decomposition): each part steps its slab plus halo layers as a periodic
 * domain and refreshes the halo layers from its neighbours after each step.
 * on_device = 0: host buffer (staged through context-owned device scratch,
 * synchronises the stream); 1: device buffer (asynchronous on the context
 * stream).  Errors: SLLBM_ERR_ARG (NULL buffer, x range outside [0, N_x)),
 * SLLBM_ERR_STATE (no state). */
int sllbm_get_x_layers(sllbm_ctx* ctx, int32_t x0, int32_t nx, void* buf, int32_t on_device);
int sllbm_set_x_layers(sllbm_ctx* ctx, int32_t x0, int32_t nx, const void* buf, int32_t on_device);

/* ------------------------------------------------------------------ stepping */

/* Advance n time steps (Eq. 1 with the boundary schemes of Sec. 3.3): one
 * fused stream + moments + collision kernel launch per step, ping-ponging the
 * two population buffers.  Asynchronous on the context stream. */
int sllbm_step(sllbm_ctx* ctx, int64_t n);

/* Number of steps taken since the last init / set_state. */
int sllbm_step_count(const sllbm_ctx* ctx, int64_t* out);

/* ------------------------------------------------------------------ forcing and control */

/* Body force density F[3] (host pointer, D components used) applied after the
 * collision with Kupershtokh's exact-difference method (Sec. 4.3):
 * f_i += f_i^eq(rho, u + du, T) - f_i^eq(rho, u, T) with du = F dt / rho; g is
 * unchanged, so momentum grows by F dt and energy by the kinetic work.
 * F = 0 switches the term off.  Takes effect from the next step. */
int sllbm_set_force(sllbm_ctx* ctx, const double* F);

/* Mass rescaling (Sec. 4.3): scale every population (f and g) by
 * target_mass / sum_n rho_n, which leaves u and T unchanged. */
int sllbm_rescale_mass(sllbm_ctx* ctx, double target_mass);

typedef struct {
    double  target_momentum;  /* target nodal mean of rho u_x                         */
    double  force0;           /* base force density F_x (e.g. rho_w Re_tau^2 mu_w^2 / delta^3) */
    double  kp, ki;           /* PI gains on the momentum error                       */
    int32_t control_every;    /* steps between force updates (0: no control)          */
    int32_t rescale_every;    /* steps between mass rescalings (0: none); Sec. 4.3 uses 10 */
    double  target_mass;      /* sum_n rho_n kept by the rescaling                    */
} sllbm_control;

/* Advance n steps with the volume force of Sec. 4.3 adjusted by a PI
 * controller on the mean streamwise momentum: every control_every steps,
 * e = target_momentum - mean(rho u_x) (FP64 reduction), I += e * control_every * dt,
 * F_x = force0 + kp e + ki I; every rescale_every steps the mass is rescaled.
 * The controller state persists in the context.  force_out (host, 3 doubles,
 * may be NULL) receives the force in effect at the end.  The reductions
 * synchronise the context stream. */
int sllbm_step_controlled(sllbm_ctx* ctx, int64_t n, const sllbm_control* control, double* force_out);

/* ------------------------------------------------------------------ readout */

/* Per-node moments (Sec. 3.1): rho[N], u[N][D], T[N] in FP64. */
int sllbm_read_moments(sllbm_ctx* ctx, double* rho, double* u, double* T, int32_t on_device);

/* Conservation sums in FP64 over all nodes: out[0] = sum rho,
 * out[1..D] = sum rho u, out[D+1] = sum (rho |u|^2 + 2 rho c_v T) (= 2 rho E).
 * Also checks positivity: returns SLLBM_ERR_UNSTABLE if any node has
 * rho <= 0 or T <= 0 or a non-finite value (out is still filled). */
int sllbm_conservation(sllbm_ctx* ctx, double* out);

/* Allocation-free variant of sllbm_conservation (the paper has no
 * counterpart; this is a service of the library).  Same sums, same outputs,
 * same SLLBM_ERR_UNSTABLE check, but the per-block partial sums live in a
 * fixed 1 MiB device array compiled into the library instead of in scratch
 * that the context allocates.  It is meant for callers that must not call
 * cudaMalloc / cudaFree at the point where they check conservation: code
 * whose device memory budget is owned by another framework's pool (a raw
 * cudaMalloc there can fail or fragment it), or a time loop that cannot
 * afford the device synchronisation a cudaFree implies.  The call allocates
 * nothing; it writes D + 2 doubles to the caller's host buffer `out`.
 *   - Limit: one partial per 256 nodes, at most 26,211 blocks in 3D
 *     (6,710,016 nodes) and 32,764 blocks in 2D (8,387,584 nodes); larger
 *     meshes get SLLBM_ERR_ARG with the limit in sllbm_last_error().
 *   - Every call looks up the array's device address (cudaGetSymbolAddress)
 *     with the context's device current, so a device reset between calls is
 *     harmless.
 *   - The call waits for the context's stream (it copies the sums and the
 *     positivity flag to the host and synchronises), so it cannot be issued
 *     while that stream is being captured into a CUDA graph.
 *   - Every call on a device shares the one array and leaves the last
 *     call's sums in it; the positivity flag is cleared at the start of each
 *     call.  Calls that overlap on the GPU (different streams or contexts of
 *     the same device at the same time) race on the array: serialise them.
 *   - Every GPU that loads the library holds the array until the process
 *     exits. */
int sllbm_conservation_static(sllbm_ctx* ctx, double* out);

/* ------------------------------------------------------------------ flow statistics */
/* Statistics of the paper's experiments, reduced on the device from the
 * moments of the current state (rho, u, T per node; p = rho T).
 *
 * Reynolds averages (Sec. 4.3, Eq. reynolds) are arithmetic means over the
 * homogeneous directions x and z, i.e. over the nodes of one plane of constant
 * y index j (N1 planes); Favre averages (Eq. favre) are mean(rho phi) /
 * mean(rho); the Reynolds stresses (Eq. rij) are
 *     R_ab = mean(rho u_a'' u_b'') / mean(rho),  u'' = u - u~.
 * Axis-aligned meshes only (box, channel, mixing layer); SLLBM_ERR_UNSUPPORTED
 * on the O-grid, SLLBM_ERR_STATE before init.  Host pointers, each may be
 * NULL: y [N1] (the plane's y coordinate), rho_bar [N1], u_bar [N1][D]
 * (Reynolds), u_favre [N1][D], T_bar [N1], p_bar [N1], R [N1][D][D]
 * (symmetric).  Synchronises the context's stream. */
int sllbm_plane_profiles(sllbm_ctx* ctx, double* y, double* rho_bar, double* u_bar, double* u_favre, double* T_bar,
                         double* p_bar, double* R);

/* Averages over time as well as over x and z (the statistics of a developed
 * channel or mixing layer): sllbm_stats_accumulate adds the current state's
 * plane means (the sums behind sllbm_plane_profiles) to running sums on the
 * device (enqueued on the context's stream, no host synchronisation);
 * sllbm_stats_reset clears them; sllbm_plane_profiles_mean derives the same
 * profiles as sllbm_plane_profiles from the time averages of those means,
 * i.e. Favre averages and Reynolds stresses over x, z and the accumulated
 * states (*samples: how many; SLLBM_ERR_STATE if none).  Axis-aligned meshes
 * only. */
int sllbm_stats_accumulate(sllbm_ctx* ctx);
int sllbm_stats_reset(sllbm_ctx* ctx);
int sllbm_plane_profiles_mean(sllbm_ctx* ctx, double* y, double* rho_bar, double* u_bar, double* u_favre,
                              double* T_bar, double* p_bar, double* R, int64_t* samples);

/* Temporal mixing layer thicknesses (Sec. 4.4) of the current state:
 *   delta_theta = 1 / (rho0 du^2) * integral over y of
 *                 rho_bar (du/2 - u1~)(du/2 + u1~) dy
 *   delta_omega = du / max |d u1_bar / dy|
 * The integral is that of the order-p Lagrange interpolant of the plane
 * values over the mesh's y cells (exact per cell); d/dy is the derivative of
 * the cell's interpolant at its nodes, maximised over every (cell, node).
 * du != 0, rho0 > 0; either output may be NULL (not both).  Axis-aligned
 * meshes only, as sllbm_plane_profiles. */
int sllbm_mixing_thickness(sllbm_ctx* ctx, double du, double rho0, double* delta_theta, double* delta_omega);

/* Pressure coefficient (Sec. 4.2) C_P = (p - p0) / (gamma/2 p0 Ma^2), p = rho T,
 * at the nodes of the plane y index 0 (side 0) or N1 - 1 (side 1): on the
 * O-grid the airfoil surface and the far-field ring, on the channel the two
 * walls.  p0 > 0 and Ma > 0 are the caller's reference (the inlet state);
 * gamma is the context's.  *count = N0 * N2 nodes (N2 = 1 in 2D), x fastest;
 * x [count][D] (node coordinates) and cp [count] are host pointers, either
 * may be NULL (both NULL: only the count, no state needed). */
int sllbm_plane_cp(sllbm_ctx* ctx, int32_t side, double p0, double mach, double* x, double* cp, int64_t* count);

/* ------------------------------------------------------------------ setup data */

/* FP64 departure records as produced by the setup pass, one per
 * (velocity i, node n), arrays [Q][N]:
 *   kind  0 interior, 1 equilibrium, 2 bounce-back, 3 isothermal bounce-back, 4 outlet
 *   src   population read (i, or opp[i] for bounce-back)
 *   bid   boundary id crossed (-1 if none)
 *   cell  departure cell (-1 for equilibrium records)
 *   xi    reference coordinates [Q][N][D]
 *   xsrc  physical source point [Q][N][D] (equals the cell map of (cell, xi))
 * Host pointers; any of them may be NULL.  For the structured mode the
 * records are expanded from the per-class records. */
int sllbm_departure_records(sllbm_ctx* ctx, int32_t* kind, int32_t* src, int32_t* bid,
                            int32_t* cell, double* xi, double* xsrc);

/* ------------------------------------------------------------------ learned collision */
/* Not in the paper: a small MLP (Q -> 64 -> 64 -> Q, tanh, BF16 weights, FP32
 * activations and accumulation) corrects the post-collision f of a coarse run.
 *   z_k = sum_i Phi_ki f^neq_i    non-equilibrium moments of the streamed state
 *                                 (Phi: weighted-orthonormal moment basis, see
 *                                 sllbm_moment_basis)
 *   x = s_in (.) z, h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), o = W3 h2 + b3
 *   delta f_i = w_i sigma (P o)_i  (P: projection off {1, xi, |xi|^2} in the
 *                                 weighted inner product -> mass, momentum and
 *                                 energy conserved exactly)
 * Available for FP32 D2Q19 contexts that run the warp-tiled structured kernel;
 * otherwise SLLBM_ERR_UNSUPPORTED. */
#define SLLBM_MLP_HIDDEN 64

/* Install (enable = 1) or disable (enable = 0) the correction.  Host
 * pointers: w_bf16 = W1[64][Q] | W2[64][64] | W3[Q][64] as bfloat16 bit
 * patterns, biases = b1[64] | b2[64] | b3[Q], s_in[Q], sigma > 0. */
int sllbm_mlp_set(sllbm_ctx* ctx, const uint16_t* w_bf16, const float* biases, const float* s_in, float sigma,
                  int32_t enable);

/* Which units evaluate the installed correction inside sllbm_step:
 *   SLLBM_MLP_TENSOR (default)  5th-generation tensor cores: per block of
 *       128 nodes three M = 128 BF16 products with FP32 accumulation in
 *       tensor memory; each FP32 activation enters as the sum of two BF16
 *       parts (hi + lo), so the result equals the CUDA-core evaluation to
 *       FP32 rounding.
 *   SLLBM_MLP_SIMT              CUDA cores, FP32 fused multiply-adds.
 * Both compute the network defined above.  Any other value: SLLBM_ERR_ARG.
 * The tensor-core kernel bounds each wait for its products (about a second);
 * if one runs out it leaves that block's f uncorrected and records
 * SLLBM_DEV_TC_TIMEOUT in the status word read by sllbm_device_status. */
#define SLLBM_MLP_TENSOR 0
#define SLLBM_MLP_SIMT   1
int sllbm_mlp_path(sllbm_ctx* ctx, int32_t path);

/* Device status word of the context: synchronises the context's stream,
 * writes the word to *code and clears it.  Host pointer.  The word is an OR
 * of bits: 0 nothing recorded; SLLBM_DEV_TC_TIMEOUT a tensor-core wait ran
 * out; SLLBM_DEV_COPY_TIMEOUT a bulk-copy wait ran out.  The SLLBM_DEV_BAD_* bits come only from the bounds-checked debug build
 * (sllbm_build_flags() & SLLBM_BUILD_CHECKED), whose step kernels test every
 * index they take from a record table or derive from one, replace an index
 * outside its range by 0 (so no access leaves its buffer; the result is then
 * wrong) and record:
 *   SLLBM_DEV_BAD_NODE  a source node outside the mesh (per axis, or relative
 *                       to the arriving node outside [0, n_nodes));
 *   SLLBM_DEV_BAD_POP   a source population outside [0, Q);
 *   SLLBM_DEV_BAD_REC   a record slot outside its table (class, tile record),
 *                       a boundary-state id outside [0, 2), or a gather-code
 *                       cell outside [0, cells);
 *   SLLBM_DEV_BAD_SMEM  a row-buffer slot outside the block's row, or a
 *                       tensor-copy destination in shared memory that is
 *                       not 128-byte aligned (the copy is skipped, and the
 *                       stage's bounded wait ends the step).
 * The paper has no counterpart: it is the substitute for a memory checker. */
#define SLLBM_DEV_TC_TIMEOUT 1
#define SLLBM_DEV_BAD_NODE   2
#define SLLBM_DEV_BAD_POP    4
#define SLLBM_DEV_BAD_REC    8
#define SLLBM_DEV_BAD_SMEM   16
#define SLLBM_DEV_COPY_TIMEOUT 32  /* a bulk-copy wait of SLLBM_STREAM_ROW_COPY ran out: that
                                      block stored nothing                                       */
int sllbm_device_status(sllbm_ctx* ctx, int32_t* code);

/* Test hook for the bounded waits: from the next launch on, every wait of the
 * tensor-core and bulk-copy kernels of this context (sllbm_mlp_path
 * SLLBM_MLP_TENSOR, SLLBM_STREAM_ROW_COPY) gives up after 2^log2_cycles SM
 * cycles instead of about 2^31, so a test can make a wait run out without
 * any fault: the kernel then records SLLBM_DEV_TC_TIMEOUT or
 * SLLBM_DEV_COPY_TIMEOUT, waits with the default bound for its own
 * operations in flight, frees its tensor memory and returns (a timed-out
 * bulk-copy block stores nothing: re-initialise the state afterwards).
 * log2_cycles = 0 restores the default; 1..31 sets the limit; anything else:
 * SLLBM_ERR_ARG.  The paper has no counterpart. */
int sllbm_debug_wait_limit(sllbm_ctx* ctx, int32_t log2_cycles);

/* How the loaded library was compiled: an OR of SLLBM_BUILD_* bits
 * (SLLBM_BUILD_CHECKED: the bounds-checked debug build, compiled with
 * -DSLLBM_CHECKED).  Needs no context and no GPU; never fails. */
#define SLLBM_BUILD_CHECKED 1
int sllbm_build_flags(void);

/* One plain step (no correction) that also writes the non-equilibrium
 * moments z [N][Q] (FP32) of the step's streamed state. */
int sllbm_step_features(sllbm_ctx* ctx, float* z, int32_t on_device);

/* Phi[Q][Q] (rows: Gram-Schmidt in sum_i w_i a_i b_i of the graded monomials
 * xi^m: total degree, then decreasing power of xi_0, then of xi_1) and the
 * projection P[Q][Q] = I - C^T G^-1 C W (C: rows 1, xi_a, |xi|^2).  Host. */
int sllbm_moment_basis(const sllbm_ctx* ctx, double* Phi, double* P);

/* Trainer of the correction on the device: FP32 master parameters
 * (flattened W1 | b1 | W2 | b2 | W3 | b3, 128 Q + 4224 + Q floats), forward
 * pass on BF16-rounded weights, loss L = (1/B) sum_samples sum_i w_i (P(o - y))_i^2,
 * Adam (0.9, 0.999, 1e-8). */
typedef struct sllbm_trainer sllbm_trainer;
int sllbm_train_create(const sllbm_ctx* ctx, const float* init_params, sllbm_trainer** out);
int sllbm_train_destroy(sllbm_trainer* tr);
const char* sllbm_train_last_error(const sllbm_trainer* tr);
/* Data: Z [M][Q] moments (sllbm_step_features) and R [M][Q] = (f_target - f_plain)/w.
 * max_degree > 0 first keeps only the moments of R (in the basis Phi) of
 * polynomial degree <= max_degree (0 keeps all).  Sets s_in_k = 1/rms(z_k)
 * (0 for moments without signal) and sigma = rms over samples of |P R|_w,
 * then stores x = s_in z and y = R / sigma. */
int sllbm_train_set_data(sllbm_trainer* tr, const float* Z, const float* R, int64_t M, int32_t max_degree,
                         int32_t on_device);
int sllbm_train_scales(const sllbm_trainer* tr, float* s_in, float* sigma);
/* One pass over the data in consecutive minibatches of `batch` samples (the
 * caller shuffles); *loss = mean minibatch loss. */
int sllbm_train_epoch(sllbm_trainer* tr, int32_t batch, float lr, float* loss);
/* Gradient (host, flattened like the parameters) and loss of the samples
 * [offset, offset + count) as one minibatch, without an update. */
int sllbm_train_grads(sllbm_trainer* tr, int64_t offset, int32_t count, float* grads, float* loss);
/* Where the trainer's forward and backward passes run: SLLBM_MLP_TENSOR
 * (default; 5th-generation tensor cores, one tile of 128 samples per block:
 * the three layers, the two backward products and the weight and bias
 * gradients as BF16 products with FP32 accumulators in tensor memory, the
 * activations and deltas split into BF16 hi and lo parts, the projection and
 * the loss on the CUDA cores) or SLLBM_MLP_SIMT (CUDA cores, FP32).  Both
 * give the same gradients to FP32 rounding; a tensor-core wait that runs out
 * makes the call that launched it fail with SLLBM_ERR_CUDA. */
int sllbm_train_path(sllbm_trainer* tr, int32_t path);
int sllbm_train_params(const sllbm_trainer* tr, float* params);
int sllbm_train_set_params(sllbm_trainer* tr, const float* params);
/* BF16 weights (layout of sllbm_mlp_set) and FP32 biases. */
int sllbm_train_export(const sllbm_trainer* tr, uint16_t* w_bf16, float* biases);

/* Synchronise the context stream. */
int sllbm_sync(sllbm_ctx* ctx);

/* cudaStream_t the context enqueues on. */
void* sllbm_stream(const sllbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SLLBM_H */
