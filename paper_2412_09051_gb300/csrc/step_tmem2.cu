// Instantiations of the row-tile kernel with two nodes per thread
// (step_tmem2.cuh): tiles of 512 arrival nodes, rows of up to 128 nodes (a
// TMA box row holds at most 256 FP32 values).
#include "step_tmem2.cuh"

namespace sllbm {

// rows of the tile along y and z for a row width: TY x TZ x NX = 512 nodes
bool rows_pairs_shape(int D, int nx, int& ty, int& tz) {
    if (D == 3) {
        if (nx == 128) { ty = 2; tz = 2; return true; }
        if (nx == 64) { ty = 4; tz = 2; return true; }
        return false;
    }
    if (nx == 128) { ty = 4; tz = 1; return true; }
    if (nx == 64) { ty = 8; tz = 1; return true; }
    return false;
}

size_t rows_pairs_smem(int D, int nx, const TmGeom2& T) {
    int ty = 0, tz = 0;
    if (!rows_pairs_shape(D, nx, ty, tz)) return 0;
    return rows_pairs_smem_bytes(T, nx, ty * tz);
}

int launch_rows_pairs(int vs, int nx, const float2* fg, float2* fgo, const void* maps, const int32_t* head,
                      const TmRec2* recs, const uint64_t* xmask, const uint64_t* smask, const float* tw,
                      const StepGeom& G, const CollideConst<float>& C, const TmGeom2& T, int* status, cudaStream_t s,
                      int grid) {
#define TPCASE(VS, NX, TY, TZ)                                                                                  \
    if (vs == VS && nx == NX)                                                                                   \
        return launch_step_rows_pairs<VS, NX, TY, TZ>(fg, fgo, maps, head, recs, xmask, smask, tw, G, C, T, status, \
                                                      s, grid);
    TPCASE(3, 128, 2, 2)
    TPCASE(3, 64, 4, 2)
    TPCASE(1, 128, 4, 1)
    TPCASE(1, 64, 8, 1)
#undef TPCASE
    return SLLBM_ERR_UNSUPPORTED;
}

}  // namespace sllbm
