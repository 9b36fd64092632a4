// FP32 instantiation of the substep kernels (the mixed-precision path: single
// precision reconstruction, fluxes, DER and constrained transport), the fused y/z
// sweeps of that path with their TMA descriptors, and its inversion fused with the
// x sweep.
#include <cudaTypedefs.h>

#include "echo_kernels.cuh"
#include "echo_sweep.cuh"
#include "echo_xsweep.cuh"

namespace echo {

template struct Path<float>;

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    }
    return fn;
}

// Cells per segment of the fused sweep along a direction of nD cells.  Automatic:
// 128 (5 recomputed halo faces per 128 cells) when the launch still fills the GPU's
// SMs four times over with 5 blocks each, else 0 -- measured on 768^3 the fused
// sweeps take 79 ms against 84 (y) and 96 (z) for the separate kernels, on 256^3
// with segments of 32 they are slower.  Forced: the longest of 128, 64, 32 that
// gives four waves, else 32 (or nD if shorter).
int sweep_segment(const Grid &g, int D, int nsm, bool forced)
{
    const int nD = D == 1 ? g.ny : g.nz, nO = D == 1 ? g.nz : g.ny;
    if (nD < 8) return 0;
    const long cols = (long)((g.nx + 31) / 32) * ((nO + 3) / 4);
    for (int T = 128; T >= (forced ? 32 : 128); T >>= 1)
        if (cols * ((nD + T - 1) / T) >= 20L * nsm) return T < nD ? T : nD;
    return forced ? (32 < nD ? 32 : nD) : 0;
}

}  // namespace

// The fused sweeps need: the staggered field with UCT and MP5 (their face data and
// reconstruction) and rows of 16-byte multiples for TMA (nx % 4 == 0); per
// direction, at least 8 cells along it and, unless forced, enough columns and
// cells for four waves of blocks (sweep_segment).
void make_sweep_maps(echo_ctx *c)
{
    const Grid &g = c->g;
    c->sweep_T[0] = c->sweep_T[1] = c->sweep_T[2] = 0;
    c->xsweep = false;
    const int mode = c->cfg.sweeps;
    if (mode == ECHO_SWEEPS_SEPARATE || !g.uct || g.rec != 0) return;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->cfg.device);
    // the inversion fused with the x sweep: rows of 8 to XS_NXMAX cells; automatic
    // where the rows give four waves of three blocks per SM
    if (g.nx >= 8 && g.nx <= XS_NXMAX &&
        (mode == ECHO_SWEEPS_FUSED || (long)g.ny * g.nz >= 12L * nsm) &&
        cudaFuncSetAttribute(k_c2p_xsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)xs_smem_bytes(XS_NXMAX)) == cudaSuccess)
        c->xsweep = true;
    cudaGetLastError();
    if (g.nx % 4 != 0) return;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 8};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4,
                                   (cuuint64_t)g.n * 4};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const cuuint32_t box_y[4] = {32, 1, 4, 8}, box_z[4] = {32, 4, 1, 8};
    for (int D = 1; D <= 2; D++) {
        const int T = sweep_segment(g, D, nsm, mode == ECHO_SWEEPS_FUSED);
        if (!T) continue;
        CUresult r = enc(&c->tm_prim[D], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->prim, dims,
                         strides, D == 1 ? box_y : box_z, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS) c->sweep_T[D] = T;
    }
}

void launch_fused_sweep(echo_ctx *c, int D, int want_amax)
{
    const Grid &g = c->g;
    const int T = c->sweep_T[D];
    const int nD = D == 1 ? g.ny : g.nz, nO = D == 1 ? g.nz : g.ny;
    const unsigned blocks =
        (unsigned)(((g.nx + 31) / 32) * ((nO + 3) / 4) * ((nD + T - 1) / T));
    float *fd = (float *)c->fdat[D];
    if (D == 1)
        launch(c, K_SWEEP_Y, k_sweep<1>, blocks, SW_COLS, 0, g, c->tm_prim[1],
               (const float *)c->prim, (const float *)c->Bf32, (float *)c->rhs, fd, c->sc, T,
               want_amax);
    else
        launch(c, K_SWEEP_Z, k_sweep<2>, blocks, SW_COLS, 0, g, c->tm_prim[2],
               (const float *)c->prim, (const float *)c->Bf32, (float *)c->rhs, fd, c->sc, T,
               want_amax);
}

void launch_c2p_xsweep(echo_ctx *c, int stage, int want_amax)
{
    const Grid &g = c->g;
    C2PParams par{c->cfg.c2p_tol, c->cfg.c2p_maxit, c->cfg.c2p_guess, 1};
    if (par.guess == ECHO_GUESS_MLP) par.guess = ECHO_GUESS_PREV;
    launch(c, K_C2P_X, k_c2p_xsweep, (unsigned)((long)g.ny * g.nz), XS_BS, xs_smem_bytes(g.nx),
           g, (const double *)c->U, (const double *)c->Bf, c->W, (float *)c->prim,
           (const float *)c->Bf32, (float *)c->rhs, (float *)c->fdat[0], par, c->sc, stage,
           want_amax);
}

}  // namespace echo
