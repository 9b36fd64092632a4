// echo_diagnostics_noalloc: the diagnostics reduction (sums of the conserved
// variables and of the face field, discrete div B, non-finite count) over arrays
// the caller already holds on the device, without allocating any device memory.
//
// Who needs it: code that must not call cudaMalloc -- for example a host program
// whose device memory is owned by a fixed-size pool or another framework, or a
// step that runs where new allocations are not allowed.  Such a caller passes its
// own device arrays and an output buffer; the block partial sums live in the
// file-scope array below instead of in memory the library would allocate.
//
// The scratch array: NA_MAX_BLOCKS partials of NA_Q = 11 doubles plus one result
// row, about 0.36 MB, held by every GPU that loads the library until the process
// exits.
// One block of 256 threads reduces 256 cells, so grids up to NA_MAX_CELLS
// (1,048,576 cells, e.g. 101^3) fit; larger grids are rejected with ECHO_ERR_ARG.
// Every call shares the array and overwrites every slot it later reads (nothing
// has to start at zero); calls that overlap on the GPU -- two streams, or two host
// threads -- race on it and must be serialised by the caller.
//
// Set-up: the first call on a device looks up the device address of the array
// with cudaGetSymbolAddress (the host-side name of a __device__ array is not a
// device address) and caches it for that device.  Make that first call before any
// stream capture.  The cached address belongs to the device's primary context: a
// caller that resets the device (cudaDeviceReset) and keeps using the library in
// the same process would find it stale, so this entry point is for processes that
// keep their primary context alive.
#include <mutex>

#include "echo_internal.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 4096;
constexpr int NA_Q = 11;  // per block: 10 sums, then max |div B|
constexpr long NA_MAX_CELLS = (long)NA_MAX_BLOCKS * NA_THREADS;
constexpr int NA_OUT = 11;  // tot[8], divb_max, divb_l2, nonfinite
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double na_scratch[NA_MAX_BLOCKS * NA_Q + 32];

std::mutex g_na_mutex;
double *g_na_ptr[NA_MAX_DEVICES] = {nullptr};

struct NaPair {
    double s, c;
};

__device__ __forceinline__ void na_add(NaPair &p, double x)
{
    double t = p.s + x;
    if (fabs(p.s) >= fabs(x)) p.c += (p.s - t) + x;
    else p.c += (x - t) + p.s;
    p.s = t;
}

// one partial per block of 256 cells: 10 plain sums (a fixed tree over the block's
// threads; the compensation happens across blocks, in k_na_final) + max |div B|
__global__ void __launch_bounds__(NA_THREADS)
k_na_partial(echo::Grid g, const double *__restrict__ U, const double *__restrict__ Bf,
             double *scratch)
{
    const long n = g.n;
    long c = blockIdx.x * (long)NA_THREADS + threadIdx.x;
    double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double dmax = 0.0;
    if (c < n) {
        int i, j, k;
        echo::coords(g, c, i, j, k);
        int bad = 0;
        for (int q = 0; q < 5; q++) {
            v[q] = U[q * n + c];
            bad += !isfinite(v[q]);
        }
        double div = 0.0;
        for (int d = 0; d < 3; d++) {
            v[5 + d] = Bf[d * n + c];
            bad += !isfinite(v[5 + d]);
            double s[6];
            for (int m = 0; m < 6; m++) s[m] = Bf[d * n + echo::shifted_rt(g, i, j, k, d, m - 3)];
            div += echo::der_c(s, g.inv_h[d], g.ho);
        }
        v[8] = div * div;
        v[9] = (double)bad;
        dmax = fabs(div);
    }
    __shared__ double sh[NA_THREADS];
    for (int q = 0; q < 10; q++) {
        sh[threadIdx.x] = v[q];
        __syncthreads();
        for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) scratch[blockIdx.x * NA_Q + q] = sh[0];
        __syncthreads();
    }
    sh[threadIdx.x] = dmax;
    __syncthreads();
    for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[blockIdx.x * NA_Q + 10] = sh[0];
}

// one thread per quantity over the nblk partials, in block order; result row after
// the partials: tot[8], divb_max, divb_l2, nonfinite
__global__ void k_na_final(double *scratch, int nblk, long n)
{
    int q = threadIdx.x;
    double *res = scratch + NA_MAX_BLOCKS * NA_Q;
    if (q < 10) {
        NaPair p{0.0, 0.0};
        for (int b = 0; b < nblk; b++) na_add(p, scratch[b * NA_Q + q]);
        double s = p.s + p.c;
        if (q < 8) res[q] = s;
        else if (q == 8) res[9] = sqrt(s / (double)n);
        else res[10] = s;
    } else if (q == 10) {
        double m = 0.0;
        for (int b = 0; b < nblk; b++) m = fmax(m, scratch[b * NA_Q + 10]);
        res[8] = m;
    }
}

// the message is what echo_last_error(NULL) returns afterwards
echo_status na_fail(echo_status st, const char *msg)
{
    echo::set_global_error(msg);
    return st;
}

}  // namespace

extern "C" {

// Declared in include/echo.h; see the comment there and at the top of this file.
echo_status echo_diagnostics_noalloc(const double *cons5, const double *bface, int nx, int ny,
                                     int nz, double lx, double ly, double lz, int ho,
                                     void *stream, double *out, int out_kind)
{
    if (nx < 1 || ny < 1 || nz < 1)
        return na_fail(ECHO_ERR_ARG, "echo_diagnostics_noalloc: grid sizes must be >= 1");
    const long n = (long)nx * ny * nz;
    if (n > NA_MAX_CELLS)
        return na_fail(ECHO_ERR_ARG,
                       "echo_diagnostics_noalloc: grid exceeds the 1048576-cell maximum of "
                       "its static scratch array");
    if (!cons5 || !bface || !out)
        return na_fail(ECHO_ERR_ARG, "echo_diagnostics_noalloc: NULL array");
    if (!(lx > 0) || !(ly > 0) || !(lz > 0) || (ho != 0 && ho != 1))
        return na_fail(ECHO_ERR_ARG, "echo_diagnostics_noalloc: bad box lengths or ho");
    if (out_kind != ECHO_PTR_HOST && out_kind != ECHO_PTR_DEVICE)
        return na_fail(ECHO_ERR_ARG, "echo_diagnostics_noalloc: bad out_kind");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
        return na_fail(ECHO_ERR_CUDA, "echo_diagnostics_noalloc: no current CUDA device");
    // the inputs (and a device output) must be device memory of the current device
    const void *ins[3] = {cons5, bface, out_kind == ECHO_PTR_DEVICE ? (const void *)out : nullptr};
    for (const void *p : ins) {
        if (!p) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeDevice ||
            a.device != dev) {
            cudaGetLastError();
            return na_fail(ECHO_ERR_ARG,
                           "echo_diagnostics_noalloc: inputs (and a device out) must be device "
                           "memory of the current device");
        }
    }
    double *scratch;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, na_scratch);
            if (e != cudaSuccess || !ptr) {
                cudaGetLastError();
                return na_fail(ECHO_ERR_CUDA,
                               "echo_diagnostics_noalloc: cudaGetSymbolAddress failed");
            }
            g_na_ptr[dev] = (double *)ptr;
        }
        scratch = g_na_ptr[dev];
    }
    echo::Grid g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.n = n;
    g.gam = 0.0;
    g.gfac = 0.0;
    g.gm1g = 0.0;
    g.gm1g32 = g.gam32 = g.gfac32 = 0.f;
    g.ho = ho;
    g.uct = 1;
    g.rec = 0;
    {
        const double h[3] = {lx / nx, ly / ny, lz / nz};
        echo::set_spacing(g, h);
    }
    g.lo[0] = g.lo[1] = g.lo[2] = 0;
    g.hi[0] = nx;
    g.hi[1] = ny;
    g.hi[2] = nz;
    g.primary = 1;
    cudaStream_t s = (cudaStream_t)stream;
    const int nblk = (int)((n + NA_THREADS - 1) / NA_THREADS);
    k_na_partial<<<nblk, NA_THREADS, 0, s>>>(g, cons5, bface, scratch);
    k_na_final<<<1, 32, 0, s>>>(scratch, nblk, n);
    cudaMemcpyKind kind = out_kind == ECHO_PTR_DEVICE ? cudaMemcpyDeviceToDevice
                                                      : cudaMemcpyDeviceToHost;
    if (cudaMemcpyAsync(out, scratch + NA_MAX_BLOCKS * NA_Q, NA_OUT * sizeof(double), kind, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return na_fail(ECHO_ERR_CUDA, "echo_diagnostics_noalloc: CUDA error");
    return ECHO_OK;
}

}  // extern "C"
