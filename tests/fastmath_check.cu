// GPU check of the FP64 path's reciprocal and reciprocal square root (rcp64, rsqrt64
// in echo_device.cuh) against CUDA's 1.0 / x and rsqrt(x): the largest difference in
// units in the last place over random doubles of every magnitude and special values.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <random>
#include <vector>

#include "echo_device.cuh"

__global__ void k_eval(const double *x, double *out, long n)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    out[4 * i + 0] = echo::rcp64(v);
    out[4 * i + 1] = 1.0 / v;
    out[4 * i + 2] = echo::rsqrt64(fabs(v));
    out[4 * i + 3] = rsqrt(fabs(v));
}

static double ulps(double a, double b)
{
    if (std::isnan(a) || std::isnan(b)) return (std::isnan(a) && std::isnan(b)) ? 0.0 : 1e300;
    if (a == b) return 0.0;
    if (std::isinf(a) || std::isinf(b)) return 1e300;
    const double u = std::ldexp(1.0, std::ilogb(b) - 52);
    return std::fabs(a - b) / u;
}

int main()
{
    const long n = 4000000;
    std::vector<double> x(n);
    std::mt19937_64 rng(2401);
    std::uniform_real_distribution<double> m(1.0, 2.0), e(-1000.0, 1000.0);
    const double special[] = {0.0, -0.0, 1.0, -1.0, 1e-310, 3e38, 3.5e38, 1e-38, 1.1e-38,
                              INFINITY, -INFINITY, NAN, 2.0, 0.5, 1e300, 1e-300};
    const long ns = sizeof(special) / sizeof(special[0]);
    for (long i = 0; i < n; i++) {
        if (i < ns) x[i] = special[i];
        else if (i % 4 == 0) x[i] = (i % 8 ? -1.0 : 1.0) * std::ldexp(m(rng), (int)e(rng));
        else x[i] = std::ldexp(m(rng), (int)(e(rng) / 50.0));  // the scheme's range
    }
    double *dx, *dout;
    cudaMalloc(&dx, n * sizeof(double));
    cudaMalloc(&dout, 4 * n * sizeof(double));
    cudaMemcpy(dx, x.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    k_eval<<<(unsigned)((n + 255) / 256), 256>>>(dx, dout, n);
    std::vector<double> out(4 * n);
    cudaMemcpy(out.data(), dout, 4 * n * sizeof(double), cudaMemcpyDeviceToHost);
    if (cudaGetLastError() != cudaSuccess) { std::printf("CUDA error\n"); return 2; }
    double mr = 0.0, ms = 0.0;
    for (long i = 0; i < n; i++) {
        mr = std::fmax(mr, ulps(out[4 * i], out[4 * i + 1]));
        ms = std::fmax(ms, ulps(out[4 * i + 2], out[4 * i + 3]));
    }
    std::printf("%ld inputs: rcp64 max %.2f ulp from 1.0/x, rsqrt64 max %.2f ulp from rsqrt\n", n,
                mr, ms);
    cudaFree(dx);
    cudaFree(dout);
    return (mr <= 2.0 && ms <= 3.0) ? 0 : 1;
}
