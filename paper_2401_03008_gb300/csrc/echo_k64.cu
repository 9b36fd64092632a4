// FP64 instantiation of the substep kernels, plus the kernels whose precision does
// not depend on the path: timestep, initialisation, diagnostics, vector-peak probe.
#include "echo_kernels.cuh"

namespace echo {

template struct Path<double>;

// ---------------------------------------------------------------------------
// timestep (Sec. 3 step 5): dt = cfl * min(h) / amax, once per step, on the device
// ---------------------------------------------------------------------------
__global__ void k_dt(Grid g, DevScalars *sc)
{
    if (sc->halt) return;
    double amax = __longlong_as_double((long long)sc->amax_bits);
    sc->amax_bits = 0ull;
    sc->amax_last = amax;
    double dt = sc->cfl * g.hmin / amax;
    if (sc->t + dt > sc->t_end) dt = sc->t_end - sc->t;
    if (!(dt > 0.0)) {
        sc->dt = 0.0;
        sc->halt |= 2;
        return;
    }
    sc->dt = dt;
    sc->t_prev = sc->t;
    sc->t = sc->t + dt;
}

void launch_dt(echo_ctx *c) { launch(c, K_DT, k_dt, 1, 1, 0, c->g, c->sc); }

// ---------------------------------------------------------------------------
// initial conserved state from primitives (Sec. 2 definitions) and the first
// warm guess W = rho h G^2
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BS)
k_init(Grid g, const double *__restrict__ prim5, const double *__restrict__ Bf,
       double *__restrict__ U, double *__restrict__ W)
{
    const long n = g.n;
    long c = blockIdx.x * (long)BS + threadIdx.x;
    if (c >= n) return;
    int i, j, k;
    coords(g, c, i, j, k);
    double s[8];
    for (int v = 0; v < 5; v++) s[v] = prim5[v * n + c];
#pragma unroll
    for (int d = 0; d < 3; d++) s[5 + d] = cell_field(g, Bf, c, i, j, k, d);
    double u[8], f[8], lm, lp;
    const double v2 = s[1] * s[1] + s[2] * s[2] + s[3] * s[3];
    phys<double, 0>(s, v2, g.gam, g.gfac, u, f, lm, lp);
    for (int v = 0; v < 5; v++) U[v * n + c] = u[v];
    W[c] = (s[0] + g.gfac * s[4]) / (1.0 - v2);
}

void launch_init(echo_ctx *c, const double *prim5)
{
    launch(c, K_INIT, k_init, nblocks(c->g.n, BS), BS, 0, c->g, prim5, (const double *)c->Bf,
           c->U, c->W);
}

void launch_curl_apot(echo_ctx *c, const double *apot)
{
    launch(c, K_CURL, k_curl<double>, nblocks(c->g.n, BS), BS, 0, c->g, apot, c->Bf, 1.0, 1);
}

// primitives in double for output: INT + C2P with the warm guess, W left untouched
void launch_prims_out(echo_ctx *c, double *out8)
{
    C2PParams par{c->cfg.c2p_tol, c->cfg.c2p_maxit, ECHO_GUESS_PREV, 0};
    launch(c, K_C2P, k_int_c2p<double, false>, nblocks(c->g.n, BS), BS, 0, c->g,
           (const double *)c->U, (const double *)c->Bf, c->W, (const MlpDev *)nullptr, out8, par,
           c->sc, 0, 0, 0);
}

__global__ void __launch_bounds__(BS)
k_copy2(long nu, long nb, double *__restrict__ du, double *__restrict__ db,
        const double *__restrict__ su, const double *__restrict__ sb)
{
    long q = blockIdx.x * (long)BS + threadIdx.x;
    if (q < nu) du[q] = su[q];
    if (q < nb) db[q] = sb[q];
}

void launch_copy_state(echo_ctx *c, double *dst_u, double *dst_b, const double *src_u,
                       const double *src_b)
{
    launch(c, K_MISC, k_copy2, nblocks(5 * c->g.n, BS), BS, 0, 5 * c->g.n, 3 * c->g.n, dst_u,
           dst_b, src_u, src_b);
}

__global__ void __launch_bounds__(BS) k_to_float(long m, const double *__restrict__ in, float *__restrict__ out)
{
    long q = blockIdx.x * (long)BS + threadIdx.x;
    if (q < m) out[q] = to_f32(in[q]);
}

void launch_bf32(echo_ctx *c)
{
    if (!c->Bf32) return;
    long m = 3 * c->g.n;
    launch(c, K_MISC, k_to_float, nblocks(m, BS), BS, 0, m, (const double *)c->Bf, c->Bf32);
}

// cold guess W0 = U for a resumed state without a stored guess
__global__ void __launch_bounds__(BS) k_w_cold(long n, const double *__restrict__ U, double *__restrict__ W)
{
    long q = blockIdx.x * (long)BS + threadIdx.x;
    if (q < n) W[q] = U[4 * n + q];
}

void launch_w_from_cold(echo_ctx *c)
{
    launch(c, K_MISC, k_w_cold, nblocks(c->g.n, BS), BS, 0, c->g.n, (const double *)c->U, c->W);
}

// ---------------------------------------------------------------------------
// diagnostics: deterministic block partials (compensated sums) + final reduction
// ---------------------------------------------------------------------------
struct Pair {
    double s, c;
};

__device__ __forceinline__ void pair_add(Pair &p, double x)
{
    double t = p.s + x;
    if (fabs(p.s) >= fabs(x)) p.c += (p.s - t) + x;
    else p.c += (x - t) + p.s;
    p.s = t;
}

__device__ __forceinline__ Pair pair_merge(Pair a, Pair b)
{
    Pair r;
    r.s = a.s;
    r.c = a.c + b.c;
    pair_add(r, b.s);
    return r;
}

constexpr int NSUM = 10;  // totals (8), div B squared, non-finite count

// mode 0: sums of the 8 state variables, sum of (div B)^2, non-finite count, max |div B|
// mode 1: sum over the grid of |a - b| (one variable)
__global__ void __launch_bounds__(DIAG_THREADS)
k_diag_partial(Grid g, const double *__restrict__ U, const double *__restrict__ Bf,
               const double *__restrict__ a, const double *__restrict__ b, double *partials,
               int mode)
{
    const long n = g.n;
    Pair acc[NSUM];
    for (int q = 0; q < NSUM; q++) acc[q] = Pair{0.0, 0.0};
    double dmax = 0.0;
    const long stride = (long)DIAG_BLOCKS * DIAG_THREADS;
    for (long c = blockIdx.x * (long)DIAG_THREADS + threadIdx.x; c < n; c += stride) {
        if (mode == 1) {
            pair_add(acc[0], fabs(a[c] - b[c]));
            continue;
        }
        int i, j, k;
        coords(g, c, i, j, k);
        int bad = 0;
        for (int v = 0; v < 5; v++) {
            double x = U[v * n + c];
            bad += !isfinite(x);
            pair_add(acc[v], x);
        }
        double div = 0.0;
        for (int d = 0; d < 3; d++) {
            double x = Bf[d * n + c];
            bad += !isfinite(x);
            pair_add(acc[5 + d], x);
            double s[6];
            for (int m = 0; m < 6; m++) s[m] = Bf[d * n + shifted_rt(g, i, j, k, d, m - 3)];
            div += der_c(s, g.inv_h[d], g.ho);
        }
        pair_add(acc[8], div * div);
        pair_add(acc[9], (double)bad);
        dmax = fmax(dmax, fabs(div));
    }
    // block reduction in a fixed tree order
    __shared__ double sh[DIAG_THREADS];
    const int nq = mode == 1 ? 1 : NSUM;
    for (int q = 0; q < nq; q++) {
        for (int part = 0; part < 2; part++) {
            // reduce s, then c, as separate compensated sums of the thread values
            sh[threadIdx.x] = part == 0 ? acc[q].s : acc[q].c;
            __syncthreads();
            for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
                if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
                __syncthreads();
            }
            if (threadIdx.x == 0) partials[blockIdx.x * DIAG_Q + 2 * q + part] = sh[0];
            __syncthreads();
        }
    }
    if (mode == 0) {
        sh[threadIdx.x] = dmax;
        __syncthreads();
        for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[blockIdx.x * DIAG_Q + 2 * NSUM] = sh[0];
    }
}

// one warp per quantity: each lane takes every 32nd block partial (compensated),
// then the lanes merge in a fixed shuffle tree, so the result does not depend on
// scheduling; the last warp takes the maximum of |div B|
__global__ void __launch_bounds__(32 * (NSUM + 1)) k_diag_final(const double *partials, double *out,
                                                                int mode)
{
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nq = mode == 1 ? 1 : NSUM;
    if (q < nq) {
        Pair p{0.0, 0.0};
        double cc = 0.0;
        for (int b = lane; b < DIAG_BLOCKS; b += 32) {
            pair_add(p, partials[b * DIAG_Q + 2 * q]);
            cc += partials[b * DIAG_Q + 2 * q + 1];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const Pair r{__shfl_down_sync(0xffffffffu, p.s, o),
                         __shfl_down_sync(0xffffffffu, p.c, o)};
            const double rc = __shfl_down_sync(0xffffffffu, cc, o);
            if (lane < o) {
                p = pair_merge(p, r);
                cc += rc;
            }
        }
        if (lane == 0) out[q] = p.s + (p.c + cc);
    } else if (mode == 0 && q == nq) {
        double m = 0.0;
        for (int b = lane; b < DIAG_BLOCKS; b += 32) m = fmax(m, partials[b * DIAG_Q + 2 * NSUM]);
        m = warp_max(m);
        if (lane == 0) out[nq] = m;
    }
}

// mode 0: out[0..9] sums, out[10] max |div B|; mode 1: out[0] = sum |a - b|
void launch_diag_mode(echo_ctx *c, int mode, const double *a, const double *b)
{
    launch(c, K_DIAG, k_diag_partial, DIAG_BLOCKS, DIAG_THREADS, 0, c->g, (const double *)c->U,
           (const double *)c->Bf, a, b, c->partials, mode);
    launch(c, K_DIAG, k_diag_final, 1, 32 * (NSUM + 1), 0, (const double *)c->partials, c->dres,
           mode);
}

// ---------------------------------------------------------------------------
// vector FMA peak probe: independent chains, no memory traffic
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T seed, T *out)
{
    T a0 = seed + threadIdx.x, a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
    T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
    const T m = T(0.999999), k = T(1e-7);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < 4; r++) {
            a0 = fma(a0, m, k); a1 = fma(a1, m, k); a2 = fma(a2, m, k); a3 = fma(a3, m, k);
            a4 = fma(a4, m, k); a5 = fma(a5, m, k); a6 = fma(a6, m, k); a7 = fma(a7, m, k);
        }
    }
    T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == T(-12345.0)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

double probe_fma_peak(echo_ctx *c, int fp64)
{
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->cfg.device);
    const int blocks = nsm * 16, threads = 256;
    void *out = nullptr;
    cudaMalloc(&out, (size_t)blocks * threads * 8);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int iters = fp64 ? 256 : 8192;
    double best = 0.0;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(e0, c->stream);
        if (fp64) k_fma_probe<double><<<blocks, threads, 0, c->stream>>>(iters, 1.0, (double *)out);
        else k_fma_probe<float><<<blocks, threads, 0, c->stream>>>(iters, 1.0f, (float *)out);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        c->launches++;
        double flops = 2.0 * 8 * 4 * (double)iters * blocks * threads;
        if (ms > 0) best = fmax(best, flops / (ms * 1e-3));
        if (ms < 20.0f) iters *= 4;  // grow until the launch is long enough to time
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return best;
}

}  // namespace echo
