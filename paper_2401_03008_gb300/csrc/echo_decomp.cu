// Block domain decomposition with a wide halo, every block on this device.
//
// Sec. 3 decomposes the periodic grid into blocks (one MPI rank each) and fills
// ghost cells before each loop that calls INT, REC or DER.  Sec. 4 and Sec. 6
// propose a halo wide enough for one exchange per substep, of all variables at
// once.  Here each block is an ordinary context over its padded extent (owned cells
// plus `halo` ghost layers per split direction); the kernels wrap periodically
// inside the padded block, which only corrupts cells within the dependency radius
// of the block's outer seam, and those are ghosts that the next exchange
// overwrites.  The blocks share one set of device scalars: the speed maximum of
// all owned faces (the allreduce(max) of a multi-rank run), one dt, one time and
// step, one failure flag that stops every block.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "echo_internal.h"

using echo::DevScalars;
using echo::nblocks;

namespace {

constexpr int BS = 256;  // threads per block of the exchange and copy kernels
char g_derr[512] = "no error";

struct Geom {
    int N[3];     // global cells per direction
    int p[3];     // blocks per direction
    int nloc[3];  // owned cells per direction
    int G[3];     // ghost layers per side (0 along an unsplit direction)
    int npad[3];  // padded extent
    long npadc;   // cells of one padded block
    long nglob;   // global cells
};

struct SubPtrs {
    double *U, *Bf, *W;
    float *Bf32;
};

}  // namespace

struct echo_decomp {
    echo_config cfg;
    Geom gm;
    int nsub;
    std::vector<echo_ctx *> sub;
    DevScalars *sc;   // shared by every block
    cudaStream_t stream;
    bool own_stream;
    SubPtrs *dsub;    // device table of the blocks' state arrays
    double *lstage;   // [11][npadc]: one block's inputs or outputs
    double *gstage;   // [11][nglob]: global host transfers (allocated on demand)
    bool has_state;
    char err[512];
};

namespace {

echo_status dfail(echo_decomp *d, echo_status st, const char *fmt, ...)
{
    char *buf = d ? d->err : g_derr;
    size_t cap = d ? sizeof(d->err) : sizeof(g_derr);
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, cap, fmt, ap);
    va_end(ap);
    return st;
}

#define DCK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return dfail(d, ECHO_ERR_CUDA, "%s: %s", #call,            \
                                            cudaGetErrorString(e_));                      \
    } while (0)

__device__ __forceinline__ int pmod(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// padded cell c of block s -> global cell index, and whether the block owns it
__device__ __forceinline__ long to_global(const Geom &gm, int s, long c, bool &own)
{
    int l[3];
    l[0] = (int)(c % gm.npad[0]);
    long r = c / gm.npad[0];
    l[1] = (int)(r % gm.npad[1]);
    l[2] = (int)(r / gm.npad[1]);
    int b[3] = {s % gm.p[0], (s / gm.p[0]) % gm.p[1], s / (gm.p[0] * gm.p[1])};
    int g[3];
    own = true;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        int x = l[d] - gm.G[d];
        if (x < 0 || x >= gm.nloc[d]) own = false;
        g[d] = pmod(b[d] * gm.nloc[d] + x, gm.N[d]);
    }
    return g[0] + (long)gm.N[0] * (g[1] + (long)gm.N[1] * g[2]);
}

// global cell -> owning block and its padded index there
__device__ __forceinline__ long to_owner(const Geom &gm, long gc, int &s)
{
    int g[3];
    g[0] = (int)(gc % gm.N[0]);
    long r = gc / gm.N[0];
    g[1] = (int)(r % gm.N[1]);
    g[2] = (int)(r / gm.N[1]);
    int b[3], l[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        b[d] = g[d] / gm.nloc[d];
        l[d] = g[d] - b[d] * gm.nloc[d] + gm.G[d];
    }
    s = b[0] + gm.p[0] * (b[1] + gm.p[1] * b[2]);
    return l[0] + (long)gm.npad[0] * (l[1] + (long)gm.npad[1] * l[2]);
}

// The halo exchange: every ghost cell of every block (blockIdx.y) takes U, the
// face field (and its float copy) and W from the block that owns it.  Reads touch
// owned cells only and writes ghost cells only, so the blocks can run together.
__global__ void __launch_bounds__(BS) k_exchange(Geom gm, const SubPtrs *__restrict__ subs)
{
    const int s = blockIdx.y;
    const long c = blockIdx.x * (long)BS + threadIdx.x;
    if (c >= gm.npadc) return;
    bool own;
    const long gc = to_global(gm, s, c, own);
    if (own) return;
    int so;
    const long oc = to_owner(gm, gc, so);
    const long np = gm.npadc;
    const SubPtrs dst = subs[s], src = subs[so];
#pragma unroll
    for (int v = 0; v < 5; v++) dst.U[v * np + c] = src.U[v * np + oc];
#pragma unroll
    for (int v = 0; v < 3; v++) {
        const double b = src.Bf[v * np + oc];
        dst.Bf[v * np + c] = b;
        if (dst.Bf32) dst.Bf32[v * np + c] = (float)b;
    }
    dst.W[c] = src.W[oc];
}

// global [ncomp][nglob] -> block s's padded [ncomp][npadc] (ghosts included)
__global__ void __launch_bounds__(BS)
k_extract(Geom gm, int s, int ncomp, const double *__restrict__ src, double *__restrict__ dst)
{
    const long c = blockIdx.x * (long)BS + threadIdx.x;
    if (c >= gm.npadc) return;
    bool own;
    const long gc = to_global(gm, s, c, own);
    for (int v = 0; v < ncomp; v++) dst[v * gm.npadc + c] = src[v * gm.nglob + gc];
}

// block s's owned cells of a padded [ncomp][npadc] -> global [ncomp][nglob]
__global__ void __launch_bounds__(BS)
k_insert(Geom gm, int s, int ncomp, const double *__restrict__ src, double *__restrict__ dst)
{
    const long c = blockIdx.x * (long)BS + threadIdx.x;
    if (c >= gm.npadc) return;
    bool own;
    const long gc = to_global(gm, s, c, own);
    if (!own) return;
    for (int v = 0; v < ncomp; v++) dst[v * gm.nglob + gc] = src[v * gm.npadc + c];
}

echo_status sync_d(echo_decomp *d)
{
    DCK(cudaGetLastError());
    DCK(cudaStreamSynchronize(d->stream));
    return ECHO_OK;
}

echo_status read_sc(echo_decomp *d, DevScalars *h)
{
    DCK(cudaMemcpyAsync(h, d->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, d->stream));
    DCK(cudaStreamSynchronize(d->stream));
    return ECHO_OK;
}

echo_status write_sc(echo_decomp *d, const DevScalars *h)
{
    DCK(cudaMemcpyAsync(d->sc, h, sizeof(DevScalars), cudaMemcpyHostToDevice, d->stream));
    DCK(cudaStreamSynchronize(d->stream));
    return ECHO_OK;
}

void exchange(echo_decomp *d)
{
    echo::Range r("halo exchange");
    dim3 grid(nblocks(d->gm.npadc, BS), d->nsub);
    k_exchange<<<grid, BS, 0, d->stream>>>(d->gm, d->dsub);
}

echo_status ensure_gstage(echo_decomp *d)
{
    if (d->gstage) return ECHO_OK;
    if (cudaMalloc((void **)&d->gstage, 11 * d->gm.nglob * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        d->gstage = nullptr;
        return dfail(d, ECHO_ERR_OOM, "global staging of %ld doubles does not fit",
                     11 * d->gm.nglob);
    }
    return ECHO_OK;
}

void free_decomp(echo_decomp *d)
{
    for (echo_ctx *c : d->sub) {
        if (!c) continue;
        c->sc = nullptr;  // shared, freed below
        echo_destroy(c);
    }
    d->sub.clear();
    if (d->sc) cudaFree(d->sc);
    if (d->dsub) cudaFree(d->dsub);
    if (d->lstage) cudaFree(d->lstage);
    if (d->gstage) cudaFree(d->gstage);
    if (d->own_stream && d->stream) cudaStreamDestroy(d->stream);
}

template <typename R>
void substep(echo_decomp *d, int stage)
{
    exchange(d);
    for (echo_ctx *c : d->sub) {
        echo::Path<R>::c2p_sweeps(c, stage, false, stage == 1);
    }
    if (stage == 1) echo::launch_dt(d->sub[0]);
    for (echo_ctx *c : d->sub) {
        echo::Path<R>::uct(c);
        echo::Path<R>::rk(c, stage);
    }
}

}  // namespace

extern "C" {

int echo_decomp_min_halo(const echo_config *cfg)
{
    if (!cfg || (cfg->uct != 0 && cfg->uct != 1) || (cfg->ho != 0 && cfg->ho != 1) ||
        (cfg->rec != ECHO_REC_MP5 && cfg->rec != ECHO_REC_LINEAR))
        return -1;
    // upwind side of the composition DER(flux(REC(C2P(INT(face field)))))
    const int der = cfg->ho ? 3 : 1;                    // faces i-5/2 or i-1/2
    const int rec = cfg->rec == ECHO_REC_MP5 ? 2 : 1;   // cells f-2 or f-1 of face f
    const int itp = cfg->uct ? (cfg->ho ? 2 : 1) : 0;   // faces i-3/2 or i-1/2
    return der + rec + itp;
}

echo_status echo_decomp_create(const echo_config *cfg, int px, int py, int pz, int halo,
                               echo_decomp **out)
{
    if (!cfg || !out) return dfail(nullptr, ECHO_ERR_ARG, "cfg or out is NULL");
    *out = nullptr;
    if (echo_decomp_min_halo(cfg) < 0) return dfail(nullptr, ECHO_ERR_ARG, "invalid scheme");
    if (cfg->c2p_guess == ECHO_GUESS_MLP)
        return dfail(nullptr, ECHO_ERR_ARG, "the learned guess is not available on blocks");
    const int N[3] = {cfg->nx, cfg->ny, cfg->nz}, P[3] = {px, py, pz};
    for (int a = 0; a < 3; a++) {
        if (N[a] < 1 || P[a] < 1 || N[a] % P[a] != 0)
            return dfail(nullptr, ECHO_ERR_ARG, "blocks per direction must divide the cells");
    }
    if (halo < 1) return dfail(nullptr, ECHO_ERR_ARG, "halo must be >= 1");
    if ((long)px * py * pz > 65535) return dfail(nullptr, ECHO_ERR_ARG, "at most 65535 blocks");
    echo_decomp *d = new echo_decomp();
    d->cfg = *cfg;
    snprintf(d->err, sizeof(d->err), "no error");
    Geom &gm = d->gm;
    gm.nglob = (long)N[0] * N[1] * N[2];
    gm.npadc = 1;
    for (int a = 0; a < 3; a++) {
        gm.N[a] = N[a];
        gm.p[a] = P[a];
        gm.nloc[a] = N[a] / P[a];
        gm.G[a] = P[a] > 1 ? halo : 0;
        gm.npad[a] = gm.nloc[a] + 2 * gm.G[a];
        gm.npadc *= gm.npad[a];
    }
    d->nsub = px * py * pz;
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        cudaGetLastError();
        delete d;
        return dfail(nullptr, ECHO_ERR_CUDA, "CUDA device %d not available", cfg->device);
    }
    if (cfg->stream) {
        d->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete d;
            return dfail(nullptr, ECHO_ERR_CUDA, "cudaStreamCreate failed");
        }
        d->own_stream = true;
    }
    const double L[3] = {cfg->lx, cfg->ly, cfg->lz};
    double h[3];
    for (int a = 0; a < 3; a++) h[a] = L[a] / N[a];  // the global cell sizes, as echo_create
    std::vector<SubPtrs> tab;
    for (int s = 0; s < d->nsub; s++) {
        echo_config sc = *cfg;
        sc.nx = gm.npad[0];
        sc.ny = gm.npad[1];
        sc.nz = gm.npad[2];
        sc.lx = h[0] * gm.npad[0];
        sc.ly = h[1] * gm.npad[1];
        sc.lz = h[2] * gm.npad[2];
        sc.stream = d->stream;
        echo_ctx *c = nullptr;
        echo_status st = echo_create(&sc, &c);
        if (st != ECHO_OK) {
            dfail(nullptr, st, "block %d: %s", s, echo_last_error(nullptr));
            free_decomp(d);
            delete d;
            return st;
        }
        d->sub.push_back(c);
        echo::set_spacing(c->g, h);
        for (int a = 0; a < 3; a++) {
            c->g.lo[a] = gm.G[a];
            c->g.hi[a] = gm.G[a] + gm.nloc[a];
        }
        c->g.primary = s == 0;
        cudaFree(c->sc);
        c->sc = nullptr;
        tab.push_back(SubPtrs{c->U, c->Bf, c->W, c->Bf32});
    }
    bool ok = cudaMalloc((void **)&d->sc, sizeof(DevScalars)) == cudaSuccess &&
              cudaMalloc((void **)&d->dsub, d->nsub * sizeof(SubPtrs)) == cudaSuccess &&
              cudaMalloc((void **)&d->lstage, 11 * gm.npadc * sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_decomp(d);
        delete d;
        return dfail(nullptr, ECHO_ERR_OOM, "block tables or staging do not fit");
    }
    for (echo_ctx *c : d->sub) c->sc = d->sc;
    DevScalars hs;
    memset(&hs, 0, sizeof(hs));
    hs.cfl = cfg->cfl;
    hs.t_end = INFINITY;
    cudaMemcpy(d->sc, &hs, sizeof(hs), cudaMemcpyHostToDevice);
    cudaMemcpy(d->dsub, tab.data(), d->nsub * sizeof(SubPtrs), cudaMemcpyHostToDevice);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        free_decomp(d);
        delete d;
        return dfail(nullptr, ECHO_ERR_CUDA, "initialisation failed");
    }
    *out = d;
    return ECHO_OK;
}

echo_status echo_decomp_destroy(echo_decomp *d)
{
    if (!d) return ECHO_OK;
    cudaSetDevice(d->cfg.device);
    cudaStreamSynchronize(d->stream);
    free_decomp(d);
    delete d;
    return ECHO_OK;
}

echo_status echo_decomp_set_state(echo_decomp *d, const double *prim, const double *bface,
                                  const double *apot, int ptr_kind)
{
    if (!d) return dfail(nullptr, ECHO_ERR_ARG, "decomp is NULL");
    if (!prim) return dfail(d, ECHO_ERR_ARG, "prim is NULL");
    if (ptr_kind != ECHO_PTR_HOST && ptr_kind != ECHO_PTR_DEVICE)
        return dfail(d, ECHO_ERR_ARG, "ptr_kind must be HOST or DEVICE");
    DCK(cudaSetDevice(d->cfg.device));
    const long N = d->gm.nglob, np = d->gm.npadc;
    const double *src[3] = {prim, bface, apot};
    const int ncomp[3] = {5, 3, 3};
    const long goff[3] = {0, 5 * N, 8 * N}, loff[3] = {0, 5 * np, 8 * np};
    if (ptr_kind == ECHO_PTR_HOST) {
        echo_status st = ensure_gstage(d);
        if (st) return st;
        for (int a = 0; a < 3; a++) {
            if (!src[a]) continue;
            DCK(cudaMemcpyAsync(d->gstage + goff[a], src[a], ncomp[a] * N * sizeof(double),
                                cudaMemcpyHostToDevice, d->stream));
            src[a] = d->gstage + goff[a];
        }
    }
    for (int s = 0; s < d->nsub; s++) {
        for (int a = 0; a < 3; a++)
            if (src[a])
                k_extract<<<nblocks(np, BS), BS, 0, d->stream>>>(d->gm, s, ncomp[a], src[a],
                                                                 d->lstage + loff[a]);
        echo_status st = echo_set_state(d->sub[s], d->lstage, bface ? d->lstage + loff[1] : nullptr,
                                        apot ? d->lstage + loff[2] : nullptr, ECHO_PTR_DEVICE);
        if (st != ECHO_OK) return dfail(d, st, "block %d: %s", s, echo_last_error(d->sub[s]));
    }
    // the padded blocks wrapped onto themselves at their seams: refill every ghost
    exchange(d);
    echo_status st = sync_d(d);
    if (st) return st;
    d->has_state = true;
    return ECHO_OK;
}

echo_status echo_decomp_step(echo_decomp *d, int max_steps, double t_end, int *steps_done,
                             double *t_now)
{
    if (!d) return dfail(nullptr, ECHO_ERR_ARG, "decomp is NULL");
    if (!d->has_state) return dfail(d, ECHO_ERR_STATE, "step before set_state");
    if (max_steps < 0) return dfail(d, ECHO_ERR_ARG, "max_steps < 0");
    DCK(cudaSetDevice(d->cfg.device));
    DevScalars h;
    echo_status st;
    if ((st = read_sc(d, &h))) return st;
    const long step0 = h.step;
    h.t_end = t_end;
    h.halt = 0;
    h.fail_stage = 0;
    h.fail_step = -1;
    if ((st = write_sc(d, &h))) return st;
    const bool mixed = d->cfg.precision == ECHO_MIXED;
    const bool finite_end = std::isfinite(t_end);
    for (int s = 0; s < max_steps; s++) {
        for (int stage = 1; stage <= d->cfg.rk_order; stage++) {
            if (mixed) substep<float>(d, stage);
            else substep<double>(d, stage);
        }
        if (finite_end) {
            if ((st = read_sc(d, &h))) return st;
            if (h.halt) break;
        }
    }
    if ((st = sync_d(d))) return st;
    if ((st = read_sc(d, &h))) return st;
    echo_status ret = ECHO_OK;
    if (h.halt & 5) {
        // bit 0: an inversion failed; bit 2: a bounded wait of the fused sweep ran out
        if (h.fail_stage >= 2) {
            for (echo_ctx *c : d->sub) {
                echo::launch_copy_state(c, c->U, c->Bf, c->U0, c->Bf0);
                echo::launch_bf32(c);
            }
            h.t = h.t_prev;
        }
        const int why = h.halt;
        h.halt = 0;
        if ((st = write_sc(d, &h))) return st;
        if ((st = sync_d(d))) return st;
        if (why & 1)
            ret = dfail(d, ECHO_ERR_C2P, "inversion failed in step %ld (stage %d, %u cells)",
                        h.fail_step, h.fail_stage, h.fails);
        else
            ret = dfail(d, ECHO_ERR_CUDA,
                        "a bounded wait for a TMA copy of the fused sweep ran out in step %ld; "
                        "the step was rolled back", h.fail_step);
    }
    if (steps_done) *steps_done = (int)(h.step - step0);
    if (t_now) *t_now = h.t;
    return ret;
}

echo_status echo_decomp_get_state(echo_decomp *d, double *cons5, double *bface, double *w,
                                  double *t, long *step, int ptr_kind)
{
    if (!d) return dfail(nullptr, ECHO_ERR_ARG, "decomp is NULL");
    if (!d->has_state) return dfail(d, ECHO_ERR_STATE, "no state");
    if (ptr_kind != ECHO_PTR_HOST && ptr_kind != ECHO_PTR_DEVICE)
        return dfail(d, ECHO_ERR_ARG, "ptr_kind must be HOST or DEVICE");
    DCK(cudaSetDevice(d->cfg.device));
    echo_status st;
    const long N = d->gm.nglob, np = d->gm.npadc;
    double *dst[3] = {cons5, bface, w};
    const int ncomp[3] = {5, 3, 1};
    for (int a = 0; a < 3; a++) {
        if (!dst[a]) continue;
        double *to = dst[a];
        if (ptr_kind == ECHO_PTR_HOST) {
            if ((st = ensure_gstage(d))) return st;
            to = d->gstage;
        }
        for (int s = 0; s < d->nsub; s++) {
            echo_ctx *c = d->sub[s];
            const double *from = a == 0 ? c->U : a == 1 ? c->Bf : c->W;
            k_insert<<<nblocks(np, BS), BS, 0, d->stream>>>(d->gm, s, ncomp[a], from, to);
        }
        if (ptr_kind == ECHO_PTR_HOST)
            DCK(cudaMemcpyAsync(dst[a], to, ncomp[a] * N * sizeof(double), cudaMemcpyDeviceToHost,
                                d->stream));
    }
    DevScalars h;
    if ((st = read_sc(d, &h))) return st;
    if (t) *t = h.t;
    if (step) *step = h.step;
    return sync_d(d);
}

echo_status echo_decomp_get_primitives(echo_decomp *d, double *out, int ptr_kind)
{
    if (!d || !out) return dfail(d, ECHO_ERR_ARG, "decomp or out is NULL");
    if (!d->has_state) return dfail(d, ECHO_ERR_STATE, "no state");
    if (ptr_kind != ECHO_PTR_HOST && ptr_kind != ECHO_PTR_DEVICE)
        return dfail(d, ECHO_ERR_ARG, "ptr_kind must be HOST or DEVICE");
    DCK(cudaSetDevice(d->cfg.device));
    echo_status st;
    double *to = out;
    if (ptr_kind == ECHO_PTR_HOST) {
        if ((st = ensure_gstage(d))) return st;
        to = d->gstage;
    }
    // the ghosts are stale after a step; INT needs the owned cells' neighbours
    exchange(d);
    for (int s = 0; s < d->nsub; s++) {
        echo::launch_prims_out(d->sub[s], d->lstage);
        k_insert<<<nblocks(d->gm.npadc, BS), BS, 0, d->stream>>>(d->gm, s, 8, d->lstage, to);
    }
    if (ptr_kind == ECHO_PTR_HOST)
        DCK(cudaMemcpyAsync(out, to, 8 * d->gm.nglob * sizeof(double), cudaMemcpyDeviceToHost,
                            d->stream));
    return sync_d(d);
}

echo_status echo_decomp_counters(echo_decomp *d, double *out)
{
    if (!d || !out) return dfail(d, ECHO_ERR_ARG, "decomp or out is NULL");
    DCK(cudaSetDevice(d->cfg.device));
    DevScalars h;
    echo_status st = read_sc(d, &h);
    if (st) return st;
    out[0] = (double)h.c2p_calls;
    out[1] = (double)h.it_sum;
    out[2] = (double)h.it_max;
    out[3] = (double)h.fails;
    out[4] = (double)h.rec_fallbacks;
    return ECHO_OK;
}

const char *echo_decomp_last_error(const echo_decomp *d) { return d ? d->err : g_derr; }

}  // extern "C"
