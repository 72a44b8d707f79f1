// Internal structures of the SLLBM library (host side + kernel argument blocks).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sllbm.h"
#include "sllbm_device.cuh"

namespace sllbm {

// record kinds (departure records)
enum { REC_INTERIOR = 0, REC_EQ = 1, REC_BB = 2, REC_BB_ISO = 3, REC_OUTLET = 4 };

// ------------------------------------------------------------ host geometry
struct HostVelSet {
    int Q = 0, D = 0;
    std::vector<double> xi;   // Q*D
    std::vector<double> w;    // Q
    std::vector<int> opp;     // Q
    std::vector<double> shell_s;   // |xi|^2 per shell (compile-time shell map)
};
int build_velocity_set(int kind, HostVelSet& vs, std::string& err);
// a caller's set (SLLBM_VELSET_CUSTOM): copied and checked (symmetry, moments to second order)
int build_custom_velocity_set(const sllbm_velset_desc& d, HostVelSet& vs, std::string& err);

// Per-velocity constants of the generic kernels (generic.cu): abscissa, the
// weights of f and g, |xi|^2 and the shell constants of the equilibrium, the
// boundary equilibria and moving-wall terms per boundary id, the opposite
// velocity.
template <typename real>
struct GenVel {
    real xi[3];
    real w, wg, s2, sA, sB, sC, sE;
    real eqf[2], eqg[2], mw[2];
    int32_t opp, pad;
};

struct HostMesh {
    int kind = 0, D = 0, p = 0;
    int cells[3] = {1, 1, 1};
    int N[3] = {1, 1, 1};
    int periodic[3] = {1, 1, 1};
    double length[3] = {1, 1, 1};
    double stretch = 1.0, thickness = 0.12;
    int central = 0;
    int64_t n_nodes = 0, n_cells = 0;
    std::vector<double> V[3];     // cell vertices per dimension (axis-aligned kinds)
    bool uniform_periodic = true; // every periodic dimension has uniform cells (class records apply)
    std::vector<double> X;        // node coordinates [N][D]
    std::vector<double> glc;      // p+1 reference nodes
};
int build_mesh(const sllbm_mesh_desc& d, HostMesh& m, std::string& err);

// ------------------------------------------------------------ device mesh view
struct MeshView {
    int kind, D, p;
    int cells[3], N[3], periodic[3];
    double length[3];
    const double* V[3];       // device vertex arrays (axis-aligned kinds)
    const double* X;          // device node coordinates (curved kinds)
    double glc[5], glc_inv_den[5];
    int bc_kind[2];
    double R;                 // NACA far-field radius
};

struct TraceArgs {            // setup kernel arguments
    MeshView M;
    double xi[SLLBM_QMAX_GENERIC][3];
    int opp[SLLBM_QMAX_GENERIC];
    int Q;
    double dt;
    int max_newton, max_walk;
};

// FP64 departure record (setup output), one per (velocity, node) or (velocity, class)
struct Rec64 {
    int32_t cell;             // linear cell, -1 for equilibrium records
    int32_t meta;             // kind | bid << 4 (bid 15 = none) | src << 8
    double xi[3];
    double xsrc[3];
};

template <typename real>
struct ClassRec {             // structured-mode record (per velocity and class)
    int32_t cell[3];          // periodic dims: offset from the home cell; else absolute
    int32_t meta;             // kind | bid << 4 | src << 8
    real wt[3][5];            // 1D Lagrange weights per dimension (p <= 4)
};

template <typename real>
struct TileRec {              // warp-tiled record (per velocity and class), 16-byte aligned
    int32_t meta;             // kind | bid << 4 | src << 8
    int32_t dxp;              // lane offsets of the 3 x taps, (dx + 8) in 4-bit fields
    int32_t dyzp;             // dy[3] (bits 0..11) and dz[3] (bits 12..23), (d + 8) in 4-bit fields
    int32_t pad0;
    int32_t rel[9];           // node offsets of the (y, z) source rows, no periodic wrap
    int32_t pad1[3];
    real rw[9];               // y x z weight products
    real wx[3];               // x weights
};

struct RowRec {               // TileRec<float> without padding, for the one-block-per-row kernel (96 B)
    int32_t meta;             // kind | bid << 4 | src << 8
    int32_t dxp;              // offsets of the 3 x taps, (dx + 8) in 4-bit fields
    int32_t dyzp;             // dy[3] (bits 0..11) and dz[3] (bits 12..23), (d + 8) in 4-bit fields
    int32_t rel[9];           // node offsets of the (y, z) source rows, no periodic wrap
    float rw[9];              // y x z weight products
    float wx[3];              // x weights
};
static_assert(sizeof(RowRec) == 96, "six 16-byte loads per record");

template <typename real, int P>
struct alignas(16) TileRecP {  // warp-tiled record of order P (per velocity and class), factorised
    int32_t meta;             // kind | bid << 4 | src << 8
    int32_t dxp;              // lane offsets of the P + 1 x taps, (dx + 8) in 4-bit fields
    int32_t dyp;              // y offsets of the P + 1 source rows, (dy + 8) in 4-bit fields
    int32_t dzp;              // z offsets, likewise (3D)
    real wx[P + 1], wy[P + 1], wz[P + 1];   // 1D Lagrange weights
};

// per (velocity, tile class, row of the tile, x parity): the streaming record
// of the rows' arrival nodes (96 bytes, staged with the source rows)
struct alignas(16) TmRec {
    int32_t meta;       // kind | bid << 4 | src << 8
    int32_t ntap;       // number of (y, z) taps (0 for equilibrium records)
    int32_t dx0;        // offset of the first of the three consecutive x taps (-2 .. 0)
    float wx[3];        // x weights
    int32_t off[9];     // byte offsets of the taps' source rows within the stage
    float w[9];         // (y, z) weight products
};
static_assert(sizeof(TmRec) == 96, "six 16-byte loads per record");

constexpr int TM_HEAD = 66;          // ints per (velocity, tile class) copy list: runs, rows, 32 runs, their first slots
constexpr int TM_MAX_RUNS = 32;
constexpr int TM_MAX_ROWS = 64;      // rows per stage
constexpr int TM_COLS = 96;          // tensor-memory columns per warp (2 Q <= 96)
constexpr int TM_ALLOC = 512;        // columns allocated per CTA (one CTA per SM)

struct TmGeom {
    int ntile_y, ntile_z, ntiles;    // tiles along y, along z, total
    int n_tc;                        // tile classes (y tiles on a non-periodic y axis, else 1)
    int nst;                         // pipeline stages
    int rows_bytes;                  // bytes of source rows per stage (max rows x NX x 8)
    int stage_bytes;                 // rows_bytes + the tile's records (+ the weight operands: tensor-core variant)
    int kp;                          // tensor-core variant: the product's K, max rows padded to 8 (else 0)
};

// one entry of a copy list: a run of `len` consecutive y rows (contiguous in
// memory) of one source population at one z, starting at y and z relative to
// the tile origin
inline constexpr int32_t tm_pack_run(int src, int dy, int dz, int len) {
    return src | ((dy + 128) << 6) | ((dz + 128) << 14) | (len << 22);
}

// Row-tile kernel with two arrival nodes per thread (step_tmem2.cuh): per
// (velocity, tile class, tile row) the record of the row's even and odd x
// nodes (128 bytes), the (y, z) taps shared by both, the x weights of each
// over a window of six row sums (x - 2 .. x + 3 of the even node x)
struct alignas(16) TmRec2 {
    int32_t meta;       // kind | bid << 4 | src << 8
    int32_t ntap;       // (y, z) taps
    int32_t off[9];     // byte offsets of the taps' source rows within the stage
    float w[9];         // (y, z) weight products
    float wxe[5];       // even node x: weights of the row sums at x - 2 .. x + 2
    float wxo[5];       // odd node x + 1: weights of the row sums at x - 1 .. x + 3
    int32_t pad[2];
};
static_assert(sizeof(TmRec2) == 128, "eight 16-byte loads per record");

// The same record at order p = 4 (352 bytes): up to 25 (y, z) taps, and the x
// weights of the two pair classes (x mod 4 = 0 and 2), each node's nine
// weights over a window of ten row sums (x - 4 .. x + 5 of the even node x)
struct alignas(16) TmRec4 {
    int32_t meta;       // kind | bid << 4 | src << 8
    int32_t ntap;       // (y, z) taps
    int32_t off[25];    // byte offsets of the taps' source rows within the stage
    float w[25];        // (y, z) weight products
    float wx[2][2][9];  // [pair class][even, odd node][row sum x - 4 + m (odd: x - 3 + m)]
};
static_assert(sizeof(TmRec4) == 352, "22 16-byte loads per record");

constexpr int TM2_MAX_BOXES = 4;     // boxes (one per source population) per (velocity, tile class)
constexpr int TM2_MAX_VEL = 6;       // velocities per stage
constexpr int TM2_HEAD = 16;         // ints per copy list: boxes, rows, per box: entry, first slot in
                                     // the stage, rows along y | along z << 8 (2 + 3 * 4 = 14); then
                                     // stage start | velocities of the stage << 8, the stage's bytes
constexpr int TM2_MAX_ROWS = 96;     // rows of one velocity's boxes
constexpr int TM2_MAX_MAPS = 32;     // box shapes (tensor maps)

struct TmGeom2 {
    int ntile_y, ntile_z, ntiles;    // tiles along y, along z, total
    int n_tc;                        // tile classes (y tiles on a non-periodic y axis, else 1)
    int nst;                         // pipeline stages: two rings (one per consumer group) of nst / 2
    int rows_bytes;                  // bytes of source rows per stage (its row capacity x NX x 8)
    int stage_bytes;                 // rows_bytes + the records of up to TM2_MAX_VEL velocities
    int rec_map;                     // index of the records' tensor map
    int ncy, ncz;                    // tile classes along y and z: class cy + ncy cz (cy = ty on a
                                     // non-periodic y axis, else ty mod ncy; cz = tz mod ncz)
    int p;                           // Lagrange order (2 or 4)
};

// one box of a copy list: population, first y and z relative to the tile
// origin, shape index (its tensor map)
inline constexpr int32_t tm2_pack_box(int src, int dy, int dz, int map) {
    return src | ((dy + 128) << 6) | ((dz + 128) << 14) | (map << 22);
}

struct StepGeom {             // structured / gather kernel geometry
    int N[3], cells[3], periodic[3];
    int ncls[3];              // classes per dimension (p if periodic, else N)
    int64_t n_nodes;
    int n_classes;
#ifdef SLLBM_CHECKED
    int* status;              // device status word of the context (bounds checks of the debug build;
                              // the release layout is kept: a longer struct changes register allocation)
#endif
};

}  // namespace sllbm

struct sllbm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string last_error;
    sllbm_mesh_desc desc{};
    sllbm_params params{};
    int velset = 0;
    sllbm::HostVelSet vs;
    sllbm::HostMesh mesh;
    int mode = SLLBM_STREAM_GATHER;      // resolved
    bool tiled = false;                  // structured mode runs the warp-tiled kernel
    bool row_copy = false;               // SLLBM_STREAM_ROW_COPY requested
    bool row_uniform = false;            // both x parities share each velocity's y/z stencil
    int tiled_p = 0;                     // order of the warp-tiled order-P table (4), 0: none
    bool want_tmem = false;              // SLLBM_STREAM_ROWS_TMEM requested
    bool want_tc = false;                // SLLBM_STREAM_TENSOR requested: (y, z) contraction on tcgen05
    float* tm_bop = nullptr;             // its weight operands [Q][n_tc][hi, lo][16 x kp] (canonical layout)
    bool rows_tmem = false;              // tables of the tensor-memory row-tile kernel built
    int tm_ty = 0, tm_tz = 0, tm_grid = 0;   // its tile shape (rows along y, z) and grid
    sllbm::TmGeom tm{};
    int32_t* tm_head = nullptr;          // copy lists [Q][n_tc][TM_HEAD]
    void* tm_recs = nullptr;             // TmRec [Q][n_tc][TY TZ][2]
    bool want_tm2 = false;               // SLLBM_STREAM_ROWS_PAIRS requested
    sllbm_alloc_fn alloc_fn = nullptr;   // caller's device allocator (sllbm_set_allocator), or cudaMalloc
    sllbm_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    bool bad_alloc = false;              // the allocator returned unusable memory (reported as an argument error)
    bool generic = false;                // a D3Q125 or caller's set: the generic kernels (generic.cu)
    void* gen_v = nullptr;               // GenVel<real> [Q] in the context's precision
    void* gen_v64 = nullptr;             // GenVel<double> [Q] (initialisation, moments, conservation)
    bool rows_tm2 = false;               // tables of the two-nodes-per-thread row-tile kernel built
    sllbm::TmGeom2 tm2{};
    int32_t* tm2_head = nullptr;         // box lists [Q][n_tc][TM2_HEAD]
    uint64_t* tm2_smask = nullptr;       // stage starts per (tile class, consumer group), bit j: velocity j
    void* tm2_recs = nullptr;            // TmRec2 [Q][n_tc][TY TZ]
    void* tm2_maps = nullptr;            // TMA tensor maps [2 state buffers][box shapes]
    std::vector<int> tm2_box;            // box shapes: rows along y | rows along z << 8
    uint64_t* tm_xmask = nullptr;        // [n_tc]: velocities whose x factor needs the row exchange
    const char* step_kernel = "";        // kernel of the last step launched (sllbm_info)
    int precision = SLLBM_FP32;
    // device geometry
    double* dV[3] = {nullptr, nullptr, nullptr};
    double* dX = nullptr;
    // FP64 setup records
    sllbm::Rec64* rec64 = nullptr;       // [Q][n_rec_units]
    int64_t n_rec_units = 0;             // nodes (gather) or classes (structured)
    // step tables
    void* cls_tab = nullptr;             // ClassRec<real>[Q][n_classes]
    void* tile_tab = nullptr;            // TileRec<real>[Q][n_classes] (warp-tiled kernel)
    void* row_tab = nullptr;             // RowRec[Q][n_classes] (one-block-per-row kernel, FP32)
    int32_t* g_code = nullptr;           // gather: [Q][N] cell | kind<<24 | bid<<28
    void* g_xi = nullptr;                // gather: real [Q][D][N]
    void* tw_tab = nullptr;              // real: per class (structured) or node (gather); NaN none
    int64_t table_bytes = 0;
    int64_t n_boundary_records = 0, n_isothermal_nodes = 0;
    // state
    void* fg[2] = {nullptr, nullptr};     // interleaved (f, g) deviations, [Q][N] pairs
    int cur = 0;
    bool initialised = false;
    int64_t steps = 0;
    // scratch
    double* d_red = nullptr;             // reduction partials
    double* d_mom = nullptr;             // scratch for host moment reads (N (D+2))
    float* mlp_img = nullptr;            // learned-collision image (device)
    std::vector<float> mlp_host;         // its host copy (constant part)
    bool mlp_enabled = false;
    bool mlp_tensor = true;              // SLLBM_MLP_TENSOR (default) or SLLBM_MLP_SIMT
    uint16_t* mlp_tc = nullptr;          // BF16 weight tiles, canonical K-major layout (device)
    int* d_status = nullptr;             // device status word (tensor-core MLP)
    double* d_plane = nullptr;           // plane statistics [N1][K]
    double* d_plane_acc = nullptr;       // running sums over time of the plane statistics
    int64_t stats_samples = 0;           // states accumulated into d_plane_acc
    double* d_cp = nullptr;              // pressure coefficient of one node plane
    double force[3] = {0.0, 0.0, 0.0};   // body force density (Kupershtokh forcing)
    double ctl_integral = 0.0;           // PI controller state
    double* d_wref = nullptr;            // reference weights w_i, w_i (2 c_v - D) for rescaling
    float* d_feat = nullptr;             // scratch for host feature reads
    void* d_layers = nullptr;            // staging of node layers read from / written to host memory
    size_t layer_bytes = 0;
    int* d_flag = nullptr;
    sllbm::StepGeom geom{};
    sllbm::CollideConst<float> cc32{};
    sllbm::CollideConst<double> cc64{};
};
