// C ABI of libecho (declared in include/echo.h): context life cycle, state
// transfer, the host stage loop of the SSP-RK3 step, diagnostics and profiling.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "echo_internal.h"

using echo::DevScalars;
using echo::Path;

namespace {

const char *kKernelNames[ECHO_NKERNELS] = {
    "int_c2p", "flux_x", "flux_y", "flux_z", "der_x", "der_y", "der_z", "uct_x",
    "uct_y", "uct_z", "rk_curl", "dt", "curl", "init", "diag", "misc", "mlp_guess",
    "sweep_y", "sweep_z", "c2p_sweep_x"};

char g_err[256] = "no error";

echo_status fail(echo_ctx *c, echo_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    if (c) vsnprintf(c->err, sizeof(c->err), fmt, ap);
    else vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(c, ECHO_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

bool is_mixed(const echo_ctx *c) { return c->cfg.precision == ECHO_MIXED; }

size_t rsize(const echo_ctx *c) { return is_mixed(c) ? sizeof(float) : sizeof(double); }

echo_status sync_check(echo_ctx *c)
{
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return ECHO_OK;
}

echo_status read_sc(echo_ctx *c, DevScalars *h)
{
    CK(cudaMemcpyAsync(h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ECHO_OK;
}

echo_status write_sc(echo_ctx *c, const DevScalars *h)
{
    CK(cudaMemcpyAsync(c->sc, h, sizeof(DevScalars), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ECHO_OK;
}

echo_status ensure_stage(echo_ctx *c)
{
    if (c->stage8) return ECHO_OK;
    if (cudaMalloc((void **)&c->stage8, 9 * c->g.n * sizeof(double)) != cudaSuccess) {
        c->stage8 = nullptr;
        cudaGetLastError();
        return fail(c, ECHO_ERR_OOM, "staging buffer of %ld doubles does not fit", 9 * c->g.n);
    }
    return ECHO_OK;
}

// device copy of a caller input: device pointers are used directly; host pointers
// are copied into the staging buffer at element offset off.
echo_status input(echo_ctx *c, const double *p, long count, int kind, long off,
                  const double **dev)
{
    if (kind == ECHO_PTR_DEVICE) {
        *dev = p;
        return ECHO_OK;
    }
    if (kind != ECHO_PTR_HOST) return fail(c, ECHO_ERR_ARG, "ptr_kind must be HOST or DEVICE");
    echo_status st = ensure_stage(c);
    if (st) return st;
    CK(cudaMemcpyAsync(c->stage8 + off, p, count * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    *dev = c->stage8 + off;
    return ECHO_OK;
}

// copy a device result to the caller (device or host)
echo_status output(echo_ctx *c, double *dst, const double *src, long count, int kind)
{
    cudaMemcpyKind k = kind == ECHO_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (dst == src) return ECHO_OK;
    CK(cudaMemcpyAsync(dst, src, count * sizeof(double), k, c->stream));
    return ECHO_OK;
}

echo_status select_device(echo_ctx *c)
{
    CK(cudaSetDevice(c->cfg.device));
    return ECHO_OK;
}

void free_all(echo_ctx *c)
{
    void *ptrs[] = {c->U, c->U0, c->Bf, c->Bf0, c->W, c->prim, c->flux, c->fdat[0], c->fdat[1],
                    c->fdat[2], c->E, c->rhs, c->sc, c->partials, c->dres, c->stage8,
                    c->mlp_w, c->guess, c->Bf32};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
    c->step_graph = nullptr;
    for (auto &r : c->prof) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    c->prof.clear();
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

}  // namespace

void echo::set_global_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

void echo::drop_step_graph(echo_ctx *c)
{
    if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
    c->step_graph = nullptr;
    c->graph_failed = false;
}

extern "C" {

echo_status echo_config_default(echo_config *cfg)
{
    if (!cfg) return fail(nullptr, ECHO_ERR_ARG, "cfg is NULL");
    memset(cfg, 0, sizeof(*cfg));
    cfg->nx = cfg->ny = cfg->nz = 32;
    cfg->lx = cfg->ly = cfg->lz = 1.0;
    cfg->gamma_ad = 4.0 / 3.0;
    cfg->cfl = 0.4;
    cfg->uct = 1;
    cfg->ho = 1;
    cfg->rec = ECHO_REC_MP5;
    cfg->precision = ECHO_FP64;
    cfg->c2p_guess = ECHO_GUESS_PREV;
    cfg->c2p_tol = 1e-6;
    cfg->c2p_maxit = 100;
    cfg->device = 0;
    cfg->stream = nullptr;
    cfg->rk_order = 3;
    cfg->sweeps = ECHO_SWEEPS_AUTO;
    return ECHO_OK;
}

echo_status echo_create(const echo_config *cfg, echo_ctx **out)
{
    if (!cfg || !out) return fail(nullptr, ECHO_ERR_ARG, "cfg or out is NULL");
    *out = nullptr;
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1)
        return fail(nullptr, ECHO_ERR_ARG, "grid sizes must be >= 1");
    if (!(cfg->lx > 0) || !(cfg->ly > 0) || !(cfg->lz > 0))
        return fail(nullptr, ECHO_ERR_ARG, "box lengths must be > 0");
    if (!(cfg->gamma_ad > 1.0)) return fail(nullptr, ECHO_ERR_ARG, "gamma_ad must be > 1");
    if (!(cfg->cfl > 0.0)) return fail(nullptr, ECHO_ERR_ARG, "cfl must be > 0");
    if (cfg->uct != 0 && cfg->uct != 1) return fail(nullptr, ECHO_ERR_ARG, "uct must be 0 or 1");
    if (cfg->ho != 0 && cfg->ho != 1) return fail(nullptr, ECHO_ERR_ARG, "ho must be 0 or 1");
    if (cfg->rec != ECHO_REC_MP5 && cfg->rec != ECHO_REC_LINEAR)
        return fail(nullptr, ECHO_ERR_ARG, "rec must be ECHO_REC_MP5 or ECHO_REC_LINEAR");
    if (cfg->rk_order != 2 && cfg->rk_order != 3)
        return fail(nullptr, ECHO_ERR_ARG, "rk_order must be 2 or 3");
    if (cfg->sweeps < ECHO_SWEEPS_AUTO || cfg->sweeps > ECHO_SWEEPS_SEPARATE)
        return fail(nullptr, ECHO_ERR_ARG, "sweeps must be ECHO_SWEEPS_AUTO, _FUSED or _SEPARATE");
    if (cfg->precision != ECHO_FP64 && cfg->precision != ECHO_MIXED)
        return fail(nullptr, ECHO_ERR_ARG, "precision must be FP64 or MIXED");
    if (cfg->c2p_guess < 0 || cfg->c2p_guess > 2)
        return fail(nullptr, ECHO_ERR_ARG, "c2p_guess out of range");
    if (!(cfg->c2p_tol > 0.0) || cfg->c2p_maxit < 1)
        return fail(nullptr, ECHO_ERR_ARG, "c2p_tol must be > 0 and c2p_maxit >= 1");
    long n = (long)cfg->nx * cfg->ny * cfg->nz;
    if (n >= (1L << 31)) return fail(nullptr, ECHO_ERR_ARG, "grid too large (>= 2^31 cells)");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, ECHO_ERR_CUDA, "CUDA device %d not available", cfg->device);
    }
    echo_ctx *c = new echo_ctx();
    memset(c->prof_count, 0, sizeof(c->prof_count));
    memset(c->prof_ms, 0, sizeof(c->prof_ms));
    c->cfg = *cfg;
    snprintf(c->err, sizeof(c->err), "no error");
    echo::Grid &g = c->g;
    g.nx = cfg->nx;
    g.ny = cfg->ny;
    g.nz = cfg->nz;
    g.n = n;
    g.gam = cfg->gamma_ad;
    g.gfac = cfg->gamma_ad / (cfg->gamma_ad - 1.0);
    g.gm1g = (cfg->gamma_ad - 1.0) / cfg->gamma_ad;
    g.gm1g32 = (float)g.gm1g;
    g.gam32 = (float)g.gam;
    g.gfac32 = (float)g.gfac;
    g.ho = cfg->ho;
    g.uct = cfg->uct;
    g.rec = cfg->rec;
    {
        const double h[3] = {cfg->lx / cfg->nx, cfg->ly / cfg->ny, cfg->lz / cfg->nz};
        echo::set_spacing(g, h);
    }
    g.lo[0] = g.lo[1] = g.lo[2] = 0;
    g.hi[0] = g.nx;
    g.hi[1] = g.ny;
    g.hi[2] = g.nz;
    g.primary = 1;
    c->mixed = cfg->precision == ECHO_MIXED;
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        delete c;
        return fail(nullptr, ECHO_ERR_CUDA, "cudaSetDevice failed");
    }
    if (cfg->stream) {
        c->stream = (cudaStream_t)cfg->stream;
        c->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(nullptr, ECHO_ERR_CUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    size_t rs = rsize(c);
    struct {
        void **p;
        size_t bytes;
    } al[] = {
        {(void **)&c->U, 5 * n * sizeof(double)},  {(void **)&c->U0, 5 * n * sizeof(double)},
        {(void **)&c->Bf, 3 * n * sizeof(double)}, {(void **)&c->Bf0, 3 * n * sizeof(double)},
        {(void **)&c->W, n * sizeof(double)},      {&c->prim, 8 * n * rs},
        {&c->flux, (cfg->uct ? 5 : 8) * n * rs},
        {&c->fdat[0], cfg->uct ? 6 * n * rs : 0},
        {&c->fdat[1], cfg->uct ? 6 * n * rs : 0},
        {&c->fdat[2], cfg->uct ? 6 * n * rs : 0},
        {&c->E, cfg->uct ? 3 * n * rs : 0},
        {&c->rhs, (cfg->uct ? 5 : 8) * n * rs},
        {(void **)&c->sc, sizeof(DevScalars)},
        {(void **)&c->partials, echo::DIAG_BLOCKS * echo::DIAG_Q * sizeof(double)},
        {(void **)&c->dres, 32 * sizeof(double)},
        {(void **)&c->Bf32, c->mixed && cfg->uct ? 3 * n * sizeof(float) : 0},
    };
    for (auto &a : al) {
        if (a.bytes == 0) continue;
        if (cudaMalloc(a.p, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            *a.p = nullptr;
            free_all(c);
            delete c;
            return fail(nullptr, ECHO_ERR_OOM, "device allocation of %zu bytes failed", a.bytes);
        }
    }
    if (c->mixed) echo::make_sweep_maps(c);
    DevScalars h;
    memset(&h, 0, sizeof(h));
    h.cfl = cfg->cfl;
    h.t_end = INFINITY;
    cudaMemcpy(c->sc, &h, sizeof(h), cudaMemcpyHostToDevice);
    cudaMemset(c->W, 0, n * sizeof(double));
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(nullptr, ECHO_ERR_CUDA, "initialisation failed");
    }
    *out = c;
    return ECHO_OK;
}

echo_status echo_destroy(echo_ctx *c)
{
    if (!c) return ECHO_OK;
    cudaSetDevice(c->cfg.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return ECHO_OK;
}

echo_status echo_set_state(echo_ctx *c, const double *prim, const double *bface,
                           const double *apot, int ptr_kind)
{
    echo::Range r("echo_set_state");
    if (!c) return fail(nullptr, ECHO_ERR_ARG, "ctx is NULL");
    if (!prim) return fail(c, ECHO_ERR_ARG, "prim is NULL");
    echo_status st = select_device(c);
    if (st) return st;
    const long n = c->g.n;
    if (bface) {
        cudaMemcpyKind k = ptr_kind == ECHO_PTR_DEVICE ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice;
        CK(cudaMemcpyAsync(c->Bf, bface, 3 * n * sizeof(double), k, c->stream));
    } else {
        CK(cudaMemsetAsync(c->Bf, 0, 3 * n * sizeof(double), c->stream));
    }
    if (apot && !c->g.uct)
        return fail(c, ECHO_ERR_ARG, "apot needs the staggered field (uct = 1)");
    if (apot) {
        const double *da;
        if ((st = input(c, apot, 3 * n, ptr_kind, 0, &da))) return st;
        echo::launch_curl_apot(c, da);
        if ((st = sync_check(c))) return st;
    }
    const double *dp;
    if ((st = input(c, prim, 5 * n, ptr_kind, 0, &dp))) return st;
    echo::launch_init(c, dp);
    echo::launch_bf32(c);
    DevScalars h;
    memset(&h, 0, sizeof(h));
    h.cfl = c->cfg.cfl;
    h.t_end = INFINITY;
    CK(cudaMemcpyAsync(c->sc, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    echo::launch_diag_mode(c, 0, nullptr, nullptr);
    double res[16];
    CK(cudaMemcpyAsync(res, c->dres, 11 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((st = sync_check(c))) return st;
    if (res[9] != 0.0) return fail(c, ECHO_ERR_NONFINITE, "initial state has non-finite values");
    c->has_state = true;
    c->w_cold = false;
    return ECHO_OK;
}

}  // extern "C"

// harvest of (features, W/U) after every inversion, for echo_mlp_harvest
struct Harvest {
    long stride, capacity;
    float *feats, *target;
    long count;  // states offered so far (slots base + q are filled while below capacity)
    long calls;
};

namespace {

template <typename R>
void launch_stage(echo_ctx *c, int stage, Harvest *hv)
{
    static const char *names[4] = {"stage", "stage 1", "stage 2", "stage 3"};
    echo::Range r(names[stage < 4 ? stage : 0]);
    // the learned guess: everywhere when selected, else for the first inversion after
    // a resume without a stored W (when the weights are loaded)
    const bool learned = c->cfg.c2p_guess == ECHO_GUESS_MLP || (stage == 1 && c->w_cold);
    if (hv) {
        Path<R>::int_c2p(c, stage, 1, learned);
        long off = (hv->calls * 7919L) % hv->stride;
        hv->count += echo::launch_mlp_harvest(c, hv->stride, off, hv->feats, hv->target,
                                              hv->count, hv->capacity);
        hv->calls++;
        Path<R>::sweeps(c, stage == 1);
    } else {
        Path<R>::c2p_sweeps(c, stage, learned, stage == 1);
    }
    if (stage == 1) c->w_cold = false;
    if (stage == 1) echo::launch_dt(c);
    Path<R>::uct(c);
    Path<R>::rk(c, stage);
}

// Capture one full step on the context's stream into c->step_graph.  A stream that
// cannot be captured (the legacy default stream, one already capturing) leaves
// graph_failed set, and the steps are launched directly.
void build_step_graph(echo_ctx *c)
{
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        c->graph_failed = true;
        return;
    }
    const long l0 = c->launches;
    for (int stage = 1; stage <= c->cfg.rk_order; stage++) {
        if (c->mixed) launch_stage<float>(c, stage, nullptr);
        else launch_stage<double>(c, stage, nullptr);
    }
    c->graph_kernels = c->launches - l0;
    c->launches = l0;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || !g || cudaGraphInstantiate(&c->step_graph, g, 0) != cudaSuccess) {
        cudaGetLastError();
        c->step_graph = nullptr;
        c->graph_failed = true;
    }
    if (g) cudaGraphDestroy(g);
}

echo_status run_steps(echo_ctx *c, int max_steps, double t_end, int *steps_done, double *t_now,
                      Harvest *hv)
{
    if (!c->has_state) return fail(c, ECHO_ERR_STATE, "echo_step before echo_set_state");
    if (max_steps < 0) return fail(c, ECHO_ERR_ARG, "max_steps < 0");
    echo_status st = select_device(c);
    if (st) return st;
    DevScalars h;
    if ((st = read_sc(c, &h))) return st;
    const long step0 = h.step;
    h.t_end = t_end;
    h.halt = 0;
    h.fail_stage = 0;
    h.fail_step = -1;
    if ((st = write_sc(c, &h))) return st;
    const bool finite_end = isfinite(t_end);
    // Without a per-step host check (no t_end, no harvest, no per-kernel timing) the
    // steps are replays of one captured step: a full step's launches as one graph
    // launch.  Every kernel reads the step state (dt, halt flag, counters) from the
    // device scalars, so the replays behave exactly like the launches.
    // A step whose first inversion starts from the learned guess because W holds no
    // previous solution is launched directly; the replays follow.
    const bool graph = !finite_end && !hv && !c->prof_on && max_steps >= 2;
    for (int s = 0; s < max_steps;) {
        if (graph && !c->w_cold) {
            if (!c->step_graph && !c->graph_failed) build_step_graph(c);
            if (c->step_graph) {
                for (; s < max_steps; s++) {
                    CK(cudaGraphLaunch(c->step_graph, c->stream));
                    c->launches += c->graph_kernels;
                }
                break;
            }
        }
        for (int stage = 1; stage <= c->cfg.rk_order; stage++) {
            if (c->mixed) launch_stage<float>(c, stage, hv);
            else launch_stage<double>(c, stage, hv);
        }
        s++;
        if (finite_end) {
            if ((st = read_sc(c, &h))) return st;
            if (h.halt) break;
        }
    }
    if ((st = sync_check(c))) return st;
    if ((st = read_sc(c, &h))) return st;
    echo_status ret = ECHO_OK;
    if (h.halt & 5) {
        // roll back to the start of the failed step (bit 0: an inversion failed;
        // bit 2: a bounded wait of the fused sweep ran out)
        if (h.fail_stage >= 2) {
            echo::launch_copy_state(c, c->U, c->Bf, c->U0, c->Bf0);
            echo::launch_bf32(c);
            h.t = h.t_prev;
        }
        const int why = h.halt;
        h.halt = 0;
        if ((st = write_sc(c, &h))) return st;
        if ((st = sync_check(c))) return st;
        if (why & 1)
            ret = fail(c, ECHO_ERR_C2P, "inversion failed in step %ld (stage %d, %u cells)",
                       h.fail_step, h.fail_stage, h.fails);
        else
            ret = fail(c, ECHO_ERR_CUDA,
                       "a bounded wait for a TMA copy of the fused sweep ran out in step %ld; "
                       "the step was rolled back", h.fail_step);
    }
    if (steps_done) *steps_done = (int)(h.step - step0);
    if (t_now) *t_now = h.t;
    return ret;
}

}  // namespace

extern "C" {

echo_status echo_step(echo_ctx *c, int max_steps, double t_end, int *steps_done, double *t_now)
{
    echo::Range r("echo_step");
    if (!c) return fail(nullptr, ECHO_ERR_ARG, "ctx is NULL");
    return run_steps(c, max_steps, t_end, steps_done, t_now, nullptr);
}

echo_status echo_mlp_harvest(echo_ctx *c, int nsteps, long stride, float *feats, float *target,
                             long capacity, long *count)
{
    if (!c) return fail(nullptr, ECHO_ERR_ARG, "ctx is NULL");
    if (!feats || !target || stride < 1 || capacity < 1)
        return fail(c, ECHO_ERR_ARG, "echo_mlp_harvest: bad buffers, stride or capacity");
    echo_status st = select_device(c);
    if (st) return st;
    Harvest hv{stride, capacity, feats, target, 0, 0};
    st = run_steps(c, nsteps, INFINITY, nullptr, nullptr, &hv);
    if (count) *count = hv.count < capacity ? hv.count : capacity;
    return st;
}

echo_status echo_rhs(echo_ctx *c, double *rhs_cons, double *rhs_face, double *amax, int ptr_kind)
{
    if (!c) return fail(nullptr, ECHO_ERR_ARG, "ctx is NULL");
    if (!c->has_state) return fail(c, ECHO_ERR_STATE, "echo_rhs before echo_set_state");
    echo_status st = select_device(c);
    if (st) return st;
    const long n = c->g.n;
    DevScalars h;
    if ((st = read_sc(c, &h))) return st;
    h.halt = 0;
    h.fail_stage = 0;
    h.amax_bits = 0;
    if ((st = write_sc(c, &h))) return st;
    double *dc = nullptr, *df = nullptr;
    if (ptr_kind == ECHO_PTR_DEVICE) {
        dc = rhs_cons;
        df = rhs_face;
    } else {
        if ((st = ensure_stage(c))) return st;
        dc = c->stage8;
        df = c->stage8 + 5 * n;
    }
    // with UCT off the rhs holds 8 components: cells [0..4], field [5..7]
    double *tmp8 = nullptr;
    if (!c->g.uct) {
        if ((st = ensure_stage(c))) return st;
        tmp8 = c->stage8;  // 8n of the 9n staging doubles
        if (ptr_kind != ECHO_PTR_DEVICE) {
            dc = c->stage8;
            df = c->stage8 + 5 * n;
        }
    }
    const bool learned = c->cfg.c2p_guess == ECHO_GUESS_MLP || c->w_cold;
    c->w_cold = false;
    if (c->mixed) {
        Path<float>::c2p_sweeps(c, 0, learned, 1);
        Path<float>::uct(c);
        if (c->g.uct) {
            if (df) Path<float>::curl_out(c, df);
            if (dc) Path<float>::rhs_out(c, dc);
        } else {
            Path<float>::rhs_out(c, tmp8);
        }
    } else {
        Path<double>::c2p_sweeps(c, 0, learned, 1);
        Path<double>::uct(c);
        if (c->g.uct) {
            if (df) Path<double>::curl_out(c, df);
            if (dc) Path<double>::rhs_out(c, dc);
        } else {
            Path<double>::rhs_out(c, tmp8);
        }
    }
    if (!c->g.uct && ptr_kind == ECHO_PTR_DEVICE) {
        if (dc) CK(cudaMemcpyAsync(dc, tmp8, 5 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        if (df) CK(cudaMemcpyAsync(df, tmp8 + 5 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
    if ((st = sync_check(c))) return st;
    if ((st = read_sc(c, &h))) return st;
    if (amax) memcpy(amax, &h.amax_bits, sizeof(double));
    const int why = h.halt;
    h.halt = 0;
    h.amax_bits = 0;
    h.fail_stage = 0;
    if ((st = write_sc(c, &h))) return st;
    if (why & 1) return fail(c, ECHO_ERR_C2P, "inversion failed in %u cells", h.fails);
    if (why & 4)
        return fail(c, ECHO_ERR_CUDA, "a bounded wait for a TMA copy of the fused sweep ran out");
    if (ptr_kind != ECHO_PTR_DEVICE) {
        if (rhs_cons && (st = output(c, rhs_cons, dc, 5 * n, ptr_kind))) return st;
        if (rhs_face && (st = output(c, rhs_face, df, 3 * n, ptr_kind))) return st;
        if ((st = sync_check(c))) return st;
    }
    return ECHO_OK;
}

echo_status echo_get_primitives(echo_ctx *c, double *out, int ptr_kind)
{
    if (!c || !out) return fail(c, ECHO_ERR_ARG, "ctx or out is NULL");
    if (!c->has_state) return fail(c, ECHO_ERR_STATE, "no state");
    echo_status st = select_device(c);
    if (st) return st;
    double *d = out;
    if (ptr_kind != ECHO_PTR_DEVICE) {
        if ((st = ensure_stage(c))) return st;
        d = c->stage8;
    }
    echo::launch_prims_out(c, d);
    if ((st = output(c, out, d, 8 * c->g.n, ptr_kind))) return st;
    return sync_check(c);
}

echo_status echo_mlp_guess(echo_ctx *c, double *out, int ptr_kind)
{
    if (!c || !out) return fail(c, ECHO_ERR_ARG, "ctx or out is NULL");
    if (!c->has_state) return fail(c, ECHO_ERR_STATE, "no state");
    if (!c->mlp_w) return fail(c, ECHO_ERR_STATE, "echo_mlp_guess before echo_mlp_load");
    echo_status st = select_device(c);
    if (st) return st;
    const long n = c->g.n;
    if (!c->guess) {
        if (cudaMalloc((void **)&c->guess, n * sizeof(double)) != cudaSuccess) {
            c->guess = nullptr;
            cudaGetLastError();
            return fail(c, ECHO_ERR_OOM, "echo_mlp_guess: %ld doubles do not fit", n);
        }
    }
    if (c->mixed) Path<float>::mlp_guess(c);
    else Path<double>::mlp_guess(c);
    if ((st = output(c, out, c->guess, n, ptr_kind))) return st;
    return sync_check(c);
}

echo_status echo_get_state(echo_ctx *c, double *cons5, double *bface, double *w, double *t,
                           long *step, int ptr_kind)
{
    if (!c) return fail(nullptr, ECHO_ERR_ARG, "ctx is NULL");
    if (!c->has_state) return fail(c, ECHO_ERR_STATE, "no state");
    echo_status st = select_device(c);
    if (st) return st;
    const long n = c->g.n;
    if (cons5 && (st = output(c, cons5, c->U, 5 * n, ptr_kind))) return st;
    if (bface && (st = output(c, bface, c->Bf, 3 * n, ptr_kind))) return st;
    if (w && (st = output(c, w, c->W, n, ptr_kind))) return st;
    DevScalars h;
    if ((st = read_sc(c, &h))) return st;
    if (t) *t = h.t;
    if (step) *step = h.step;
    return sync_check(c);
}

echo_status echo_set_conserved(echo_ctx *c, const double *cons5, const double *bface,
                               const double *w, double t, long step, int ptr_kind)
{
    if (!c || !cons5 || !bface) return fail(c, ECHO_ERR_ARG, "ctx, cons5 or bface is NULL");
    echo_status st = select_device(c);
    if (st) return st;
    const long n = c->g.n;
    cudaMemcpyKind k = ptr_kind == ECHO_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(c->U, cons5, 5 * n * sizeof(double), k, c->stream));
    CK(cudaMemcpyAsync(c->Bf, bface, 3 * n * sizeof(double), k, c->stream));
    if (w) CK(cudaMemcpyAsync(c->W, w, n * sizeof(double), k, c->stream));
    else echo::launch_w_from_cold(c);
    c->w_cold = w == nullptr;
    echo::launch_bf32(c);
    DevScalars h;
    if ((st = read_sc(c, &h))) return st;
    memset(&h, 0, sizeof(h));
    h.cfl = c->cfg.cfl;
    h.t_end = INFINITY;
    h.t = t;
    h.step = step;
    if ((st = write_sc(c, &h))) return st;
    c->has_state = true;
    return sync_check(c);
}

echo_status echo_diagnostics(echo_ctx *c, echo_diag *out, int reset_counters)
{
    echo::Range r("echo_diagnostics");
    if (!c || !out) return fail(c, ECHO_ERR_ARG, "ctx or out is NULL");
    if (!c->has_state) return fail(c, ECHO_ERR_STATE, "no state");
    echo_status st = select_device(c);
    if (st) return st;
    echo::launch_diag_mode(c, 0, nullptr, nullptr);
    double res[16];
    CK(cudaMemcpyAsync(res, c->dres, 11 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    DevScalars h;
    if ((st = read_sc(c, &h))) return st;
    memset(out, 0, sizeof(*out));
    out->t = h.t;
    out->dt = h.dt;
    out->amax = h.amax_last;
    for (int v = 0; v < 8; v++) out->tot[v] = res[v];
    out->divb_l2 = sqrt(res[8] / (double)c->g.n);
    out->nonfinite = (long)res[9];
    out->divb_max = res[10];
    out->c2p_calls = (long)h.c2p_calls;
    out->newton_it_mean = h.c2p_calls ? (double)h.it_sum / (double)h.c2p_calls : 0.0;
    out->newton_it_max = (int)h.it_max;
    out->newton_it32_mean = h.c2p_calls ? (double)h.it32_sum / (double)h.c2p_calls : 0.0;
    out->c2p_fallbacks = h.fallbacks;
    out->c2p_failures = h.fails;
    out->step = h.step;
    if (reset_counters) {
        h.it_sum = 0;
        h.it32_sum = 0;
        h.c2p_calls = 0;
        h.it_max = 0;
        h.fallbacks = 0;
        h.fails = 0;
        h.rec_fallbacks = 0;
        if ((st = write_sc(c, &h))) return st;
    }
    return sync_check(c);
}

echo_status echo_l1_error(echo_ctx *c, const double *ref, int ptr_kind, double *out)
{
    if (!c || !ref || !out) return fail(c, ECHO_ERR_ARG, "ctx, ref or out is NULL");
    if (!c->has_state) return fail(c, ECHO_ERR_STATE, "no state");
    echo_status st = select_device(c);
    if (st) return st;
    if ((st = ensure_stage(c))) return st;
    const long n = c->g.n;
    echo::launch_prims_out(c, c->stage8);
    for (int v = 0; v < 8; v++) {
        const double *dr;
        if ((st = input(c, ref + v * n, n, ptr_kind, 8 * n, &dr))) return st;
        echo::launch_diag_mode(c, 1, c->stage8 + v * n, dr);
        double s;
        CK(cudaMemcpyAsync(&s, c->dres, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if ((st = sync_check(c))) return st;
        out[v] = s / (double)n;
    }
    return ECHO_OK;
}

echo_status echo_profile_enable(echo_ctx *c, int on)
{
    if (!c) return fail(nullptr, ECHO_ERR_ARG, "ctx is NULL");
    c->prof_on = on != 0;
    return ECHO_OK;
}

echo_status echo_profile_read(echo_ctx *c, int k, long *launches, double *ms, const char **name,
                              int reset)
{
    if (!c || k < 0 || k >= ECHO_NKERNELS) return fail(c, ECHO_ERR_ARG, "bad kernel index");
    echo_status st = select_device(c);
    if (st) return st;
    if (!c->prof.empty()) {
        CK(cudaStreamSynchronize(c->stream));
        for (auto &r : c->prof) {
            float t = 0.f;
            cudaEventElapsedTime(&t, r.e0, r.e1);
            c->prof_count[r.kind]++;
            c->prof_ms[r.kind] += t;
            cudaEventDestroy(r.e0);
            cudaEventDestroy(r.e1);
        }
        c->prof.clear();
    }
    if (launches) *launches = c->prof_count[k];
    if (ms) *ms = c->prof_ms[k];
    if (name) *name = kKernelNames[k];
    if (reset) {
        c->prof_count[k] = 0;
        c->prof_ms[k] = 0.0;
    }
    return ECHO_OK;
}

long echo_launches(const echo_ctx *c) { return c ? c->launches : 0; }

echo_status echo_probe_fma_peak(echo_ctx *c, int precision, double *flops)
{
    if (!c || !flops) return fail(c, ECHO_ERR_ARG, "ctx or flops is NULL");
    echo_status st = select_device(c);
    if (st) return st;
    *flops = echo::probe_fma_peak(c, precision == ECHO_FP64);
    return sync_check(c);
}

void *echo_stream(const echo_ctx *c) { return c ? (void *)c->stream : nullptr; }

const char *echo_last_error(const echo_ctx *c) { return c ? c->err : g_err; }

}  // extern "C"
