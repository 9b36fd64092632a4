/*
 * echo.h -- C ABI of libecho: the per-timestep right-hand-side update of the ECHO
 * special-relativistic MHD scheme (arXiv 2401.03008) on a periodic 3-D Cartesian
 * grid, computed by hand-written CUDA kernels for sm_103a (NVIDIA GB300).
 *
 * What one step computes (Sec. 3, the five numbered steps of one Runge-Kutta
 * substep, applied to the flat-space ideal-MHD system of Sec. 2, Eq. 8):
 *   1. INT of the staggered field to cell centres and the Newton inversion of
 *      conserved to primitive variables (C2P);
 *   2. MP5 reconstruction of primitives at every interface, physical fluxes,
 *      fast speeds and the HLL flux;
 *   3. DER of the numerical fluxes into the right-hand side (Eq. 9);
 *   4. UCT edge electric fields and their curl (Eq. 10), which keeps the discrete
 *      div B at round-off;
 *   5. the SSP-RK3 stage combination; the timestep from the largest fast speed,
 *      once per full step.
 *
 * Conventions shared by every entry point
 *   - Grid arrays are float64, structure of arrays, [var][nz][ny][nx] with x
 *     fastest, periodic, no ghost cells.  Cell (i,j,k) is centred at
 *     ((i+1/2)hx, (j+1/2)hy, (k+1/2)hz) with h = L/n per direction.
 *   - Face array d, index (i,j,k): the face half a cell above the centre of cell
 *     (i,j,k) along d (Bx at (i+1/2, j, k), ...).  Edge array c, index (i,j,k): the
 *     edge half a cell above the centre along both directions other than c
 *     (Ax at (i, j+1/2, k+1/2), ...).
 *   - ptr_kind: ECHO_PTR_HOST for host memory (copied synchronously), or
 *     ECHO_PTR_DEVICE for device memory of the context's device (for example a
 *     torch tensor's data_ptr()); device pointers must stay valid until the call
 *     returns.  Input buffers are caller-owned and only read; output buffers are
 *     caller-allocated and fully overwritten.
 *   - Every call returns an echo_status.  Nothing aborts, traps or prints.  The
 *     text of the last error of a context is available from echo_last_error().
 *   - A context is used by one host thread at a time.  All state lives in the
 *     context, except the text of the last error of a call made without one
 *     (static buffers: echo_last_error(NULL), echo_decomp_last_error(NULL)) and the
 *     fixed scratch array of echo_diagnostics_noalloc.
 */
#ifndef ECHO_H
#define ECHO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct echo_ctx echo_ctx; /* opaque; created and owned by the library */

typedef enum {
    ECHO_OK = 0,
    ECHO_ERR_ARG = -1,       /* invalid argument or configuration */
    ECHO_ERR_CUDA = -2,      /* a CUDA runtime call failed */
    ECHO_ERR_OOM = -3,       /* device allocation failed */
    ECHO_ERR_C2P = -4,       /* Newton inversion failed somewhere; state rolled back */
    ECHO_ERR_NONFINITE = -5, /* non-finite value in the state; state rolled back */
    ECHO_ERR_STATE = -6      /* call out of order (for example step before set_state) */
} echo_status;

enum { ECHO_PTR_HOST = 0, ECHO_PTR_DEVICE = 1 };
/* ECHO_REC_MP5: the five-point MP5 scheme (Sec. 3); ECHO_REC_LINEAR: linear
 * reconstruction with the monotonized-central limiter (the faster variant of Sec. 4,
 * usually with rk_order = 2). */
enum { ECHO_REC_MP5 = 0, ECHO_REC_LINEAR = 1 };
/* ECHO_FP64: every step in double precision.  ECHO_MIXED: reconstruction, fluxes,
 * HLL, DER and the UCT fields in single precision; the inversion (Lorentz factor and
 * pressure recovery included) and the Runge-Kutta accumulation of the conserved
 * state in double precision.  The mixed path refines each Newton starting guess
 * with FP32 iterations, then takes FP64 chord steps (FP64 residual, the FP32
 * slope) and stops after the first undamped one with |dW| <= c2p_tol W, whose
 * remaining error is below about 1e-5 c2p_tol W. */
enum { ECHO_FP64 = 0, ECHO_MIXED = 1 };
/* Newton starting guess: W of the previous call at the same cell, W0 = U, or the
 * small learned network loaded with echo_mlp_load (falls back to the previous W
 * where its guess is unusable). */
enum { ECHO_GUESS_PREV = 0, ECHO_GUESS_COLD = 1, ECHO_GUESS_MLP = 2 };
/* Kernels of the mixed path's substep (Sec. 3 steps 1-3).  Along y and z the fused
 * kernel stages planes of the primitives in shared memory by TMA and keeps the face
 * fluxes on chip (REC, fluxes, HLL and DER in one pass); along x the fused kernel
 * is the inversion (INT + C2P) of a row of cells followed by the row's REC, fluxes,
 * HLL and DER from shared memory.  The separate kernels invert every cell, then
 * write the fluxes of one direction and take their DER in a second kernel.  Both
 * compute the same arithmetic per cell and face, compiled apart, so they agree to
 * FP32 rounding, not bit for bit.  ECHO_SWEEPS_AUTO: fused where it pays (grids of
 * at least four waves of blocks); ECHO_SWEEPS_FUSED: fused wherever the grid allows
 * it; ECHO_SWEEPS_SEPARATE: never.  The fused kernels need UCT and MP5; the y/z one
 * also nx a multiple of 4 (rows of 16-byte multiples for TMA) and at least 8 cells
 * along its direction, the x one 8 <= nx <= 1024.  The x one is not used with the
 * learned guess or a harvest.  Elsewhere, and on the FP64 path, the separate kernels
 * run. */
enum { ECHO_SWEEPS_AUTO = 0, ECHO_SWEEPS_FUSED = 1, ECHO_SWEEPS_SEPARATE = 2 };

typedef struct {
    int nx, ny, nz;     /* cells per direction, periodic; each >= 1 */
    double lx, ly, lz;  /* box lengths (> 0) */
    double gamma_ad;    /* adiabatic index of the ideal-gas law (Sec. 2, Eq. 6) */
    double cfl;         /* dt = cfl * min(h) / max fast speed (Sec. 3 step 5) */
    int uct;            /* 1: staggered field evolved by UCT (Sec. 3, Eq. 10); 0: the field is
                           cell-centred like the other variables and all 8 components take
                           the HLL flux (Sec. 3: UCT off; div B is then not preserved) */
    int ho;             /* 1: fourth-order INT and sixth-order DER; 0: two-point forms */
    int rec;            /* ECHO_REC_MP5 or ECHO_REC_LINEAR (also used inside UCT) */
    int precision;      /* ECHO_FP64 or ECHO_MIXED */
    int c2p_guess;      /* ECHO_GUESS_* */
    double c2p_tol;     /* Newton stop: an undamped step |dW| <= tol W, then one polishing
                           step (FP64 path; the mixed path stops at that step) */
    int c2p_maxit;      /* Newton iteration cap (a cell past it is a failure) */
    int device;         /* CUDA device ordinal */
    void *stream;       /* cudaStream_t to launch on; NULL: the library makes one */
    int rk_order;       /* 3: SSP-RK3 (default); 2: SSP-RK2 (the faster variant of Sec. 4) */
    int sweeps;         /* ECHO_SWEEPS_*: the mixed path's fused or separate sweep kernels */
} echo_config;

/* Fill *cfg with defaults: 32^3 unit box, gamma 4/3, cfl 0.4, uct 1, ho 1, MP5,
 * FP64, previous-W guess, tol 1e-6, maxit 100, device 0, own stream, SSP-RK3,
 * ECHO_SWEEPS_AUTO. */
echo_status echo_config_default(echo_config *cfg);

/* Validate cfg, select its device, allocate the device state (library-owned) and
 * return a context in *out.  ECHO_ERR_ARG for an invalid configuration,
 * ECHO_ERR_OOM when the device memory does not fit. */
echo_status echo_create(const echo_config *cfg, echo_ctx **out);

/* Free everything the context owns.  NULL is accepted. */
echo_status echo_destroy(echo_ctx *ctx);

/* Initial data (Sec. 4 and Sec. 5 set up the state from primitives and field).
 *   prim  [5][nz][ny][nx]: rho, vx, vy, vz, p at cell centres (required);
 *   bface [3][nz][ny][nx]: staggered field on faces (NULL: zero); with uct = 0 the
 *         cell-centred field;
 *   apot  [3][nz][ny][nx]: edge vector potential (NULL: none; uct = 1 only); its
 *         discrete curl, with the same DER as the induction equation, is added to
 *         bface so that the discrete div B is zero to round-off.
 * The conserved variables follow from the definitions of Sec. 2 (D = rho G,
 * S = rho h G^2 v + E x B, U = rho h G^2 - p + (E^2+B^2)/2, E = -v x B) with the
 * cell-centred field from INT.  Resets t and the step count to 0.  ECHO_ERR_ARG for
 * a NULL prim; ECHO_ERR_NONFINITE if the resulting state is not finite. */
echo_status echo_set_state(echo_ctx *ctx, const double *prim, const double *bface,
                           const double *apot, int ptr_kind);

/* Advance by Runge-Kutta steps (SSP-RK3, or SSP-RK2 with rk_order = 2; Sec. 3,
 * steps 1-5) until max_steps steps are done or t reaches t_end (the last step is
 * shortened to land on t_end; pass
 * INFINITY for no limit).  *steps_done and *t_now (either may be NULL) receive
 * the steps taken and the time reached.  On ECHO_ERR_C2P or ECHO_ERR_NONFINITE the
 * state, t and the step count are those at the start of the step that failed; so
 * too on ECHO_ERR_CUDA from a bounded wait of the mixed path's fused sweep that ran
 * out (a TMA copy that did not arrive).
 * Without t_end (and without kernel timing) the first call captures one full step
 * as a CUDA graph on the context's stream and every step replays it.  The call
 * synchronises its stream before returning, so it cannot itself be captured into a
 * caller's graph. */
echo_status echo_step(echo_ctx *ctx, int max_steps, double t_end, int *steps_done,
                      double *t_now);

/* Evaluate the right-hand side L(U) of Eq. 9-10 once on the current state
 * (Sec. 3 steps 1-4) without advancing it.
 *   rhs_cons [5][nz][ny][nx]: dD/dt, dS/dt, dU/dt at cell centres;
 *   rhs_face [3][nz][ny][nx]: dB/dt on faces;
 *   amax: the largest HLL speed over all faces (may be NULL).
 * The warm Newton guess is updated as a step would.  ECHO_ERR_C2P if the inversion
 * failed somewhere (the outputs are then not meaningful). */
echo_status echo_rhs(echo_ctx *ctx, double *rhs_cons, double *rhs_face, double *amax,
                     int ptr_kind);

/* Primitives for output: [8][nz][ny][nx] = rho, vx, vy, vz, p, Bx, By, Bz with the
 * field at cell centres (INT) -- Sec. 3 step 1 applied to the current state. */
echo_status echo_get_primitives(echo_ctx *ctx, double *out, int ptr_kind);

/* Checkpoint: the conserved state cons5 [5][nz][ny][nx] (D, Sx, Sy, Sz, U), the
 * staggered field bface [3][nz][ny][nx], the warm Newton guess w [nz][ny][nx],
 * t and the step count.  Any output pointer may be NULL. */
echo_status echo_get_state(echo_ctx *ctx, double *cons5, double *bface, double *w,
                           double *t, long *step, int ptr_kind);

/* Resume from a checkpoint written by echo_get_state (same layouts).  w may be NULL:
 * the first inversion then starts from the learned guess if one is loaded
 * (echo_mlp_load), else from W0 = U.  A resumed run with w is bit-identical to an
 * uninterrupted one. */
echo_status echo_set_conserved(echo_ctx *ctx, const double *cons5, const double *bface,
                               const double *w, double t, long step, int ptr_kind);

typedef struct {
    double t, dt, amax;        /* time, last dt, largest fast speed of the last step */
    double divb_max, divb_l2;  /* discrete div B (same DER as the curl), max |.| and RMS */
    double tot[8];             /* sums of D, Sx, Sy, Sz, U and face Bx, By, Bz (compensated) */
    double newton_it_mean;     /* FP64 Newton iterations per inversion since the last reset */
    int newton_it_max;
    long c2p_calls, c2p_fallbacks, c2p_failures;
    long nonfinite;            /* non-finite values found in the state */
    long step;
    double newton_it32_mean;   /* FP32 pre-iterations per inversion (mixed path) */
} echo_diag;

/* Diagnostics of the current state (Sec. 3: div B preserved by UCT; conservation of
 * the periodic-box totals).  Reductions run in a fixed order, so the result is
 * deterministic.  reset_counters != 0 clears the Newton counters afterwards. */
echo_status echo_diagnostics(echo_ctx *ctx, echo_diag *out, int reset_counters);

/* L1 norm per variable of (current primitives - ref) over the grid, divided by the
 * cell count: ref [8][nz][ny][nx] in the layout of echo_get_primitives, out[8]. */
echo_status echo_l1_error(echo_ctx *ctx, const double *ref, int ptr_kind, double *out);

/* Kernel timing for the benchmark: when enabled, every kernel launch of the
 * context is bracketed by CUDA events on the context's stream.  echo_profile_read
 * returns, for kernel kind k (0 <= k < ECHO_NKERNELS), its launch count and summed
 * device time in ms, and its name in *name; the counters are then cleared when
 * reset != 0.  echo_launches returns the number of kernels launched so far. */
#define ECHO_NKERNELS 20
echo_status echo_profile_enable(echo_ctx *ctx, int on);
echo_status echo_profile_read(echo_ctx *ctx, int k, long *launches, double *ms,
                              const char **name, int reset);
long echo_launches(const echo_ctx *ctx);

/* Measured vector peak (the roofline denominator of ALU-bound kernels): runs an
 * independent-FMA-chain kernel on the context's device and returns FLOP/s in
 * *flops (an FMA counts as 2).  precision: ECHO_FP64 or ECHO_MIXED (= FP32). */
echo_status echo_probe_fma_peak(echo_ctx *ctx, int precision, double *flops);

/* ---- The learned Newton starting guess (a service of this library; the paper
 * has no learned component).  Network 5 -> 64 -> 64 -> 1 with tanh hidden layers
 * on five rotation-invariant, dimensionless features of a cell's conserved state
 * (D/U, S^2/U^2, B^2/U, (S.B)^2/(S^2 B^2), ln(U/D)); output y = W/U and guess
 * W0 = U y.  Parameters: a flat float array of ECHO_MLP_NPARAM values in the order
 * W1[64][5], b1[64], W2[64][64], b2[64], w3[64], b3.  The 64x64 products run as
 * BF16 tensor-core MMAs with FP32 accumulation.  The Newton iteration always runs
 * to tolerance: the guess changes iteration counts, and results only within that
 * tolerance. ---- */
#define ECHO_MLP_NPARAM 4609

typedef struct {
    int epochs;          /* passes over the data */
    int batch;           /* minibatch size, a multiple of 64 */
    double lr, beta1, beta2, eps;  /* Adam */
    double lr_decay;     /* learning rate multiplied by this after every epoch */
    unsigned long seed;  /* offset of the per-epoch batch permutation */
} echo_train_cfg;

/* Load parameters (host, n = ECHO_MLP_NPARAM floats) into the context.  The
 * inversion then starts Newton from the learned guess, computed inside the
 * inversion kernel, at every cell when c2p_guess = ECHO_GUESS_MLP, and in any case
 * for the first inversion after echo_set_conserved without a stored W (where no
 * previous solution exists).  Cells whose guess is unusable fall back to the
 * previous W and are counted (echo_diag.c2p_fallbacks). */
echo_status echo_mlp_load(echo_ctx *ctx, const float *weights, long n);

/* The learned guess W0 = U y of every cell for the current state, out [nz][ny][nx]
 * (host or device, ptr_kind): the value the inversion starts from when it uses the
 * network (the same device code).  ECHO_ERR_STATE before echo_mlp_load or
 * echo_set_state; allocates n doubles on the first call. */
echo_status echo_mlp_guess(echo_ctx *ctx, double *out, int ptr_kind);

/* Inference on its own: y[n] (device) for features feats[n][5] (device) with the
 * parameters weights (host), on stream (NULL: default stream). */
echo_status echo_mlp_forward(const float *weights, const float *feats, long n, float *y,
                             void *stream);

/* Mean squared loss of y against target[n] (device) and its gradient grad[4609]
 * (host) for parameters weights (host) over the n samples feats[n][5] (device);
 * n a multiple of 64.  Same kernels as training. */
echo_status echo_mlp_grad(const float *weights, const float *feats, const float *target, long n,
                          float *grad, float *loss, void *stream);

/* Train with Adam on the GPU: feats[n][5], target[n] (device, e.g. from
 * echo_mlp_harvest); weights (host) hold the initial parameters on entry and the
 * trained ones on exit; loss_hist[epochs] (host, may be NULL) the mean loss of
 * each epoch. */
echo_status echo_mlp_train(const float *feats, const float *target, long n,
                           const echo_train_cfg *cfg, float *weights, float *loss_hist,
                           void *stream);

/* Advance nsteps SSP-RK3 steps (as echo_step) and, after every inversion, append the
 * features and the converged W/U of every stride-th cell (cells offset + q stride,
 * the offset rotating between inversions) to feats[capacity][5] and
 * target[capacity] (device): in cell order within an inversion and in inversion
 * order across them, so the buffers are deterministic.  *count receives the number
 * of states written (at most capacity). */
echo_status echo_mlp_harvest(echo_ctx *ctx, int nsteps, long stride, float *feats, float *target,
                             long capacity, long *count);

/* Diagnostics without any device allocation, for callers that cannot allocate.
 * The paper has no counterpart: this is a service of the library.  Some callers
 * must not call cudaMalloc (their device memory belongs to a fixed pool or to
 * another framework, or new allocations are not allowed where they run); they
 * still hold the state on the device and want its health checks.  This call
 * computes, over the caller's own device arrays, what echo_diagnostics reports
 * about a state: out[0..7] = sums of D, Sx, Sy, Sz, U and face Bx, By, Bz,
 * out[8] = max |div B|, out[9] = RMS div B, out[10] = number of non-finite values.
 *   cons5 [5][nz][ny][nx] and bface [3][nz][ny][nx]: device memory of the current
 *         device, in the layouts of echo_get_state; only read.
 *   nx, ny, nz, lx, ly, lz, ho: the grid, as in echo_config.
 *   stream: cudaStream_t to run on (NULL: the default stream); the call returns
 *         after the stream has finished the reduction.
 *   out: 11 doubles, host (out_kind = ECHO_PTR_HOST) or device memory of the
 *         current device (ECHO_PTR_DEVICE).
 * No memory is allocated: the block partial sums live in a fixed array of about
 * 0.36 MB inside the library, which every GPU that loads the library holds until
 * the process exits.  It limits the grid to 1,048,576 cells; larger grids return
 * ECHO_ERR_ARG.  Every call shares that array, so calls that overlap on the GPU
 * (several streams or host threads at once) race and must be serialised by the
 * caller.  The first call on a device looks up the array's device address and
 * keeps it for the process (it belongs to the device's primary context, which must
 * not be reset in between); make that first call before any stream capture.
 * Errors: ECHO_ERR_ARG (sizes, NULL, non-device inputs, or a non-device out with
 * ECHO_PTR_DEVICE), ECHO_ERR_CUDA; the text is in echo_last_error(NULL).  The sums agree
 * with echo_diagnostics to rounding (the summation order differs). */
echo_status echo_diagnostics_noalloc(const double *cons5, const double *bface, int nx,
                                     int ny, int nz, double lx, double ly, double lz, int ho,
                                     void *stream, double *out, int out_kind);

/* ---------------------------------------------------------------------------
 * Block domain decomposition with a wide halo, all subdomains on one device.
 *
 * Sec. 3 splits the periodic grid into blocks, one MPI rank each, and fills ghost
 * cells before every loop that calls INT, REC or DER; Sec. 4 and Sec. 6 propose
 * instead a halo wide enough that one exchange per Runge-Kutta substep, of all
 * variables at once, serves the whole substep.  This object is that plan with the
 * ranks kept on one GPU: the grid of cfg is split into px * py * pz equal blocks,
 * each stored as a padded block with `halo` ghost cells on both sides of every
 * split direction (none along an unsplit one, which stays periodic on itself).
 * Before each substep one exchange copies, for every ghost cell of every block, U
 * (5), the face field (3) and the Newton guess W from the block that owns the
 * cell; each block then runs the single-grid substep kernels on its padded
 * extent, and only its owned cells are kept.  The step's speed
 * maximum is taken over the owned faces of all blocks (the allreduce(max) of a
 * multi-rank run), so every block takes the same dt.  With halo >=
 * echo_decomp_min_halo(cfg) the owned cells come out bit-identical to those of one
 * undecomposed context with the same cfg; a narrower halo lets the blocks' seams
 * reach them.  The blocks share one stream (cfg->stream, or one the object
 * creates); the learned guess is not available here (ECHO_ERR_ARG). */
typedef struct echo_decomp echo_decomp;

/* The dependency radius, in cells, of one substep on the exchanged data: the DER
 * stencil (3 faces with HO, 1 without), the REC stencil (2 cells for MP5, 1 for
 * linear) and the INT stencil (2 faces with HO, 1 without, 0 without UCT), summed
 * over the upwind side.  Returns -1 for a NULL or invalid cfg. */
int echo_decomp_min_halo(const echo_config *cfg);

/* cfg: the global grid and scheme, as for echo_create.  px, py, pz >= 1 blocks per
 * direction, each dividing the cells of its direction; halo >= 1 ghost cells.
 * Errors: ECHO_ERR_ARG, ECHO_ERR_OOM, ECHO_ERR_CUDA (text in
 * echo_decomp_last_error(NULL)). */
echo_status echo_decomp_create(const echo_config *cfg, int px, int py, int pz, int halo,
                               echo_decomp **out);
echo_status echo_decomp_destroy(echo_decomp *d);

/* Global arrays in the layouts of echo_set_state, host or device (ptr_kind). */
echo_status echo_decomp_set_state(echo_decomp *d, const double *prim, const double *bface,
                                  const double *apot, int ptr_kind);

/* As echo_step, on all blocks; on ECHO_ERR_C2P every block returns to the start of
 * the failed step. */
echo_status echo_decomp_step(echo_decomp *d, int max_steps, double t_end, int *steps_done,
                             double *t_now);

/* Global outputs assembled from the owned cells, in the layouts of echo_get_state
 * and echo_get_primitives (any of cons5, bface, w, t, step may be NULL). */
echo_status echo_decomp_get_state(echo_decomp *d, double *cons5, double *bface, double *w,
                                  double *t, long *step, int ptr_kind);
echo_status echo_decomp_get_primitives(echo_decomp *d, double *out, int ptr_kind);

/* Inversion statistics of the owned cells of all blocks since set_state:
 * out[0] = inversions, out[1] = FP64 Newton iterations summed, out[2] = largest
 * iteration count, out[3] = failed inversions, out[4] = interface states reset
 * to first order. */
echo_status echo_decomp_counters(echo_decomp *d, double *out);

/* Text of the last error on d (a static string when d is NULL). */
const char *echo_decomp_last_error(const echo_decomp *d);

/* The context's stream (cudaStream_t) and device. */
void *echo_stream(const echo_ctx *ctx);

/* Text of the last error on ctx (a static string when ctx is NULL). */
const char *echo_last_error(const echo_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* ECHO_H */
