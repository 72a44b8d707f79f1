// Instantiations of the row-tile kernel with two nodes per thread
// (step_tmem2.cuh): tiles of 256 arrival nodes in 3D (two CTAs per SM) and of
// 512 in 2D (one CTA per SM), rows of up to 128 nodes (a TMA box row holds at
// most 256 FP32 values); orders 2 (3D and 2D) and 4 (3D).
#include "step_tmem2.cuh"

namespace sllbm {

// rows of the tile along y and z for a row width and order: TY x TZ x NX =
// 256 nodes in 3D, 512 in 2D.  At order 4 a tile is one z row deep: a node on a cell boundary
// and its neighbour take departure cells one apart, so a tile's source rows
// span up to 9 rows along each dimension it covers with more than one row
bool rows_pairs_shape(int D, int nx, int p, int& ty, int& tz) {
    if (p == 4) {
        // 256 nodes, two CTAs per SM; one stage per ring (boxes of up to 9 x 5 rows)
        if (D != 3) return false;
        if (nx == 128) { ty = 2; tz = 1; return true; }
        if (nx == 64) { ty = 4; tz = 1; return true; }
        return false;
    }
    if (D == 3) {
        // tiles of 256 nodes, two CTAs per SM: one CTA's collision overlaps
        // the other's streaming
        if (nx == 128) { ty = 2; tz = 1; return true; }
        if (nx == 64) { ty = 2; tz = 2; return true; }
        return false;
    }
    if (nx == 128) { ty = 4; tz = 1; return true; }
    if (nx == 64) { ty = 8; tz = 1; return true; }
    return false;
}

int launch_rows_pairs(int vs, int nx, const float2* fg, float2* fgo, const void* maps, const int32_t* head,
                      const void* recs, const uint64_t* xmask, const uint64_t* smask, const float* tw,
                      const StepGeom& G, const CollideConst<float>& C, const TmGeom2& T, int* status, cudaStream_t s,
                      int grid) {
#define TPCASE(VS, NX, TY, TZ, P)                                                                              \
    if (vs == VS && nx == NX && T.p == P)                                                                     \
        return launch_step_rows_pairs<VS, NX, TY, TZ, P>(fg, fgo, maps, head, recs, xmask, smask, tw, G, C, T, \
                                                         status, s, grid);
    TPCASE(3, 128, 2, 1, 2)
    TPCASE(3, 64, 2, 2, 2)
    TPCASE(1, 128, 4, 1, 2)
    TPCASE(1, 64, 8, 1, 2)
    TPCASE(3, 128, 2, 1, 4)
    TPCASE(3, 64, 4, 1, 4)
#undef TPCASE
    return SLLBM_ERR_UNSUPPORTED;
}

}  // namespace sllbm
