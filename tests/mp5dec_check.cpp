// Host check of the FP32-decided MP5 smooth test (echo_mp5dec.cuh) against the same
// test evaluated in FP64: on every input where mp5_test32 decides, its answer must
// be the FP64 one.  Prints the counts and exits non-zero on any mismatch.
#include <cmath>
#include <cstdio>
#include <random>

#include "echo_mp5dec.cuh"

static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

int main()
{
    std::mt19937_64 rng(240103008);
    std::uniform_real_distribution<double> u(-1.0, 1.0), lg(-12.0, 8.0), sm(-1e-3, 1e-3);
    long n = 0, undecided = 0, bad = 0, smooth = 0;
    auto check = [&](double um2, double um1, double u0, double up1, double up2) {
        const double d = 0.0234375 * um2 - 0.15625 * um1 - 0.296875 * u0 + 0.46875 * up1 -
                         0.0390625 * up2;
        const double t = d * (d - minmod(up1 - u0, 4.0 * (u0 - um1)));
        const int ref = t <= 1e-10 ? 1 : 0;
        const int got = echo::mp5_test32(d, um1, u0, up1);
        ++n;
        smooth += ref;
        if (got < 0) ++undecided;
        else if (got != ref) {
            if (bad < 10)
                std::printf("mismatch: %.17g %.17g %.17g %.17g %.17g t=%.17g\n", um2, um1, u0,
                            up1, up2, t);
            ++bad;
        }
    };
    // smooth data of every scale: a cubic sampled with a random spacing
    for (int q = 0; q < 4000000; q++) {
        const double s = std::pow(10.0, lg(rng)), h = std::pow(10.0, -3.0 * std::fabs(u(rng)));
        const double c0 = s * u(rng), c1 = s * u(rng), c2 = s * u(rng), c3 = s * u(rng);
        double v[5];
        for (int m = 0; m < 5; m++) {
            const double x = (m - 2) * h;
            v[m] = c0 + x * (c1 + x * (c2 + x * c3));
        }
        check(v[0], v[1], v[2], v[3], v[4]);
    }
    // rough data: independent values, also with a large common offset
    for (int q = 0; q < 4000000; q++) {
        const double s = std::pow(10.0, lg(rng)), off = (q & 1) ? 0.0 : s * 1e4 * u(rng);
        check(off + s * u(rng), off + s * u(rng), off + s * u(rng), off + s * u(rng),
              off + s * u(rng));
    }
    // near the threshold: small perturbations around values whose t is close to 1e-10
    for (int q = 0; q < 4000000; q++) {
        const double a = std::pow(10.0, -5.0 + 0.5 * u(rng));
        const double base = 10.0 * u(rng);
        const double v1 = base + a * u(rng), v2 = base + a * u(rng), v3 = base + a * u(rng);
        check(base + a * u(rng), v1, v2, v3, base + a * u(rng));
    }
    // exact zeros, uniform values, tiny magnitudes, one nonzero value
    for (int q = 0; q < 1000000; q++) {
        const double s = std::pow(10.0, -300.0 * std::fabs(u(rng)));
        double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        const int k = q % 6;
        if (k < 5) v[k] = s * u(rng);
        const double c = (q & 8) ? 1.0 : 0.0;
        check(c + v[0], c + v[1], c + v[2], c + v[3], c + v[4]);
    }
    std::printf("%ld inputs, %ld smooth, %ld undecided (%.3f %%), %ld mismatches\n", n, smooth,
                undecided, 100.0 * undecided / n, bad);
    return bad ? 1 : 0;
}
