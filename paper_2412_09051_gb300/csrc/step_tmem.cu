// Instantiations of the tensor-memory row-tile step kernel (step_tmem.cuh)
// for the row widths it is built for, each as a tile of 512 arrival nodes.
#include "step_tmem.cuh"

namespace sllbm {

// rows of the tile along y and z for a row width: TY x TZ x NX = 512 nodes
bool rows_tmem_shape(int D, int nx, int& ty, int& tz) {
    if (D == 3) {
        if (nx == 128) { ty = 2; tz = 2; return true; }
        if (nx == 64) { ty = 4; tz = 2; return true; }
        if (nx == 32) { ty = 4; tz = 4; return true; }
        return false;
    }
    if (nx == 256) { ty = 2; tz = 1; return true; }
    if (nx == 128) { ty = 4; tz = 1; return true; }
    if (nx == 64) { ty = 8; tz = 1; return true; }
    if (nx == 32) { ty = 16; tz = 1; return true; }
    return false;
}

size_t rows_tmem_smem_bytes(int D, int nx, const TmGeom& T) {
    int ty = 0, tz = 0;
    if (!rows_tmem_shape(D, nx, ty, tz)) return 0;
    size_t b = size_t(T.nst) * T.stage_bytes + sizeof(float2) * 2 * ty * tz * (nx + 4) +
               sizeof(uint64_t) * (2 * T.nst + 1) + 16;
    if (T.kp) b = (b + 1023) / 1024 * 1024 + 4 * size_t(nx) * T.kp * 4 + 8;   // A operands, MMA barrier
    return b < 120 * 1024 ? 120 * 1024 : b;
}

int launch_rows_tmem(int vs, int nx, const float2* fg, float2* fgo, const float* bop, const int32_t* head,
                     const TmRec* recs, const uint64_t* xmask, const float* tw, const StepGeom& G,
                     const CollideConst<float>& C, const TmGeom& T, int* status, cudaStream_t s, int grid) {
#define TMCASE(VS, NX, TY, TZ) \
    if (vs == VS && nx == NX)  \
        return launch_step_rows_tmem<VS, NX, TY, TZ, false>(fg, fgo, bop, head, recs, xmask, tw, G, C, T, status, s, grid);
    if (T.kp) {
        if (vs == 3 && nx == 128)
            return launch_step_rows_tmem<3, 128, 2, 2, true>(fg, fgo, bop, head, recs, xmask, tw, G, C, T, status, s,
                                                             grid);
        return SLLBM_ERR_UNSUPPORTED;
    }
    TMCASE(3, 128, 2, 2)
    TMCASE(3, 64, 4, 2)
    TMCASE(3, 32, 4, 4)
    TMCASE(1, 256, 2, 1)
    TMCASE(1, 128, 4, 1)
    TMCASE(1, 64, 8, 1)
    TMCASE(1, 32, 16, 1)
#undef TMCASE
    return SLLBM_ERR_UNSUPPORTED;
}

}  // namespace sllbm
