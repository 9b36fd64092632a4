// Host-side context of libecho (shared by the API and the kernel translation units).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "../../include/echo.h"
#include "echo_device.cuh"

namespace echo {

// kernel kinds for launch counting and event timing
enum Kind {
    K_C2P = 0, K_FLUX_X, K_FLUX_Y, K_FLUX_Z, K_DER_X, K_DER_Y, K_DER_Z,
    K_UCT_X, K_UCT_Y, K_UCT_Z, K_RK, K_DT, K_CURL, K_INIT, K_DIAG, K_MISC, K_MLP,
    K_SWEEP_Y, K_SWEEP_Z, K_C2P_X
};

struct ProfRec {
    int kind;
    cudaEvent_t e0, e1;
};

}  // namespace echo

struct echo_ctx {
    echo_config cfg;
    echo::Grid g;
    cudaStream_t stream;
    bool own_stream;
    int mixed;

    // conserved state (double): U[5n], U0[5n], Bf[3n], Bf0[3n]; warm guess W[n]
    double *U, *U0, *Bf, *Bf0, *W;
    float *Bf32;    // mixed path: float copy of the face field read by the sweeps
    // work buffers in the reconstruction precision R (double or float)
    void *prim;     // [8][n]  rho, vx, vy, vz, p, Bx, By, Bz at centres
    void *flux;     // [5][n]  HLL flux of one direction
    void *fdat[3];  // [6][n]  per direction: vL_d, vL_d+1, vR_d, vR_d+1, a+, a-
    void *E;        // [3][n]  edge fields
    void *rhs;      // [5][n]  cell right-hand side
    echo::DevScalars *sc;   // device scalars
    double *partials;       // reduction scratch of the diagnostics
    double *dres;           // reduction results (device)
    double *stage8;         // staging for host outputs [8][n] (allocated on demand)
    void *mlp_w;            // learned-guess weights in their device form, or NULL
    double *guess;          // learned guesses [n] for echo_mlp_guess (allocated on demand)
    // W holds no previous solution (a checkpoint resumed without it: W = U); the
    // next inversion starts from the learned guess if the weights are loaded
    bool w_cold;

    bool has_state;
    long launches;
    bool prof_on;
    // one full step captured as a CUDA graph and replayed for runs without a
    // per-step host check (see run_steps); rebuilt when the launch set changes
    cudaGraphExec_t step_graph;
    long graph_kernels;     // kernels in one replay (for the launch count)
    bool graph_failed;      // capture not possible on this stream: launch directly
    unsigned mlp_blocks;    // persistent grid of the learned-guess kernel (0: not loaded)
    // mixed path: TMA descriptors of the float primitive array for the fused y and z
    // sweeps (index 1, 2) and their segment lengths (0: that direction takes the
    // separate flux and DER kernels)
    CUtensorMap tm_prim[3];
    int sweep_T[3];
    // mixed path: the inversion and the x sweep as one kernel (k_c2p_xsweep)
    bool xsweep;
    std::vector<echo::ProfRec> prof;
    long prof_count[ECHO_NKERNELS];
    double prof_ms[ECHO_NKERNELS];
    char err[512];
};

namespace echo {

// Launch helper: counts launches and, when profiling, brackets with events.
template <typename Kernel, typename... Args>
inline void launch(echo_ctx *c, int kind, Kernel k, dim3 grid, dim3 block, size_t smem,
                   Args... args)
{
    ProfRec r;
    if (c->prof_on) {
        r.kind = kind;
        cudaEventCreate(&r.e0);
        cudaEventCreate(&r.e1);
        cudaEventRecord(r.e0, c->stream);
    }
    k<<<grid, block, smem, c->stream>>>(args...);
    if (c->prof_on) {
        cudaEventRecord(r.e1, c->stream);
        c->prof.push_back(r);
    }
    c->launches++;
}

inline unsigned nblocks(long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// NVTX range for the host phases (a step, a stage, set-up, diagnostics, the halo
// exchange): a profiler attached to the process shows them on its timeline; without
// one the calls return at once.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// Number of blocks of the fixed-shape reductions (a multiple of the SM count of
// the GB300, 152, so the partial sums have a fixed order).
constexpr int DIAG_BLOCKS = 608;
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_Q = 24;  // quantities per block partial

// Per-precision kernel launchers (one translation unit per precision).
template <typename R>
struct Path {
    // INT + C2P into the work prims (R).  stage: 1..3 (0 for a one-off call);
    // update_w: store the converged W as the next warm guess; learned: start Newton
    // from the learned guess (computed in the kernel) when the weights are loaded.
    static void int_c2p(echo_ctx *c, int stage, int update_w, bool learned);
    // the learned guesses of the current state into c->guess (echo_mlp_guess)
    static void mlp_guess(echo_ctx *c);
    // sweeps + DER (steps 2-3), want_amax on the first stage of a step; with_x = 0
    // leaves out the x sweep (done with the inversion by k_c2p_xsweep)
    static void sweeps(echo_ctx *c, int want_amax, int with_x = 1);
    // INT + C2P (updating W) and the sweeps of one substep: on the mixed path the
    // inversion and the x sweep as one kernel where the context chose it (not with
    // the learned guess), else int_c2p then sweeps
    static void c2p_sweeps(echo_ctx *c, int stage, bool learned, int want_amax);
    // UCT edge fields (step 4, first half)
    static void uct(echo_ctx *c);
    // RK stage with the curl of E (step 4, second half, and step 5)
    static void rk(echo_ctx *c, int stage);
    // curl of the work E into a face array: out = -curl E (as in dB/dt)
    static void curl_out(echo_ctx *c, double *out);
    // copy the work rhs (R) to a double array
    static void rhs_out(echo_ctx *c, double *out);
    // blocks of the persistent learned-guess kernel that fit on the device at once
    static unsigned mlp_grid(echo_ctx *c);
};

// precision-independent launchers (FP64 translation unit)
void launch_dt(echo_ctx *c);
void launch_init(echo_ctx *c, const double *prim5);
void launch_curl_apot(echo_ctx *c, const double *apot);
void launch_prims_out(echo_ctx *c, double *out8);
// mode 0: state sums, div B, non-finite count into dres[0..10]; mode 1: sum |a - b| into dres[0]
void launch_diag_mode(echo_ctx *c, int mode, const double *a, const double *b);
void launch_copy_state(echo_ctx *c, double *dst_u, double *dst_b, const double *src_u,
                       const double *src_b);
void launch_w_from_cold(echo_ctx *c);
// refresh the float copy of the face field (mixed path) after the state changed
void launch_bf32(echo_ctx *c);
double probe_fma_peak(echo_ctx *c, int fp64);
// error text of calls without a context (returned by echo_last_error(NULL))
void set_global_error(const char *msg);
// drop the captured step graph (the launch set changed)
void drop_step_graph(echo_ctx *c);
// mixed path: choose the y/z sweep kernels (cfg.sweeps and the grid) and build the
// TMA descriptors of the fused ones (c->sweep_T)
void make_sweep_maps(echo_ctx *c);
// mixed path: the fused reconstruction + flux + DER sweep along D = 1, 2
void launch_fused_sweep(echo_ctx *c, int D, int want_amax);
// mixed path: INT + C2P fused with the x sweep (c->xsweep)
void launch_c2p_xsweep(echo_ctx *c, int stage, int want_amax);
// harvest of training states (features, converged W/U) of cells offset + q stride
// into slots base + q (those below capacity); returns the number of such cells
long launch_mlp_harvest(echo_ctx *c, long stride, long offset, float *feats, float *target,
                        long base, long capacity);

}  // namespace echo
