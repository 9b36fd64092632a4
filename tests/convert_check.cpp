// Host check of the integer-pipe float <-> double conversions of the library
// against the host's IEEE conversions (round to nearest even).  Prints the
// number of mismatches per class and exits non-zero on any.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <random>

#include "echo_convert.cuh"

static bool same64(double a, double b)
{
    if (std::isnan(a) && std::isnan(b)) return echo::bits64(a) == echo::bits64(b);
    return echo::bits64(a) == echo::bits64(b);
}

int main()
{
    long bad_w = 0, bad_n = 0, n_w = 0, n_n = 0;
    // widening: every 5th float bit pattern, plus every pattern below 2^24
    // (zero and the subnormals)
    for (uint64_t b = 0; b < (1ull << 32); b += (b < (1u << 24) ? 1 : 5)) {
        const float x = echo::from_bits32((uint32_t)b);
        const double ref = (double)x;
        const double got = echo::to_f64(x);
        ++n_w;
        if (std::isnan(ref) ? !std::isnan(got) : !same64(ref, got)) ++bad_w;
    }
    // narrowing: random bit patterns, values near the float range limits, and
    // exact ties between neighbouring floats
    std::mt19937_64 rng(2401);
    auto check = [&](double x) {
        const float ref = (float)x, got = echo::to_f32(x);
        ++n_n;
        if (std::isnan(ref) ? !std::isnan(got) : echo::bits32(ref) != echo::bits32(got)) ++bad_n;
    };
    for (int q = 0; q < 20000000; q++) check(echo::from_bits64(rng()));
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    for (int q = 0; q < 5000000; q++) {
        const int ex = (int)(rng() % 300) - 150;
        check(std::ldexp(u(rng), ex));
    }
    for (int q = 0; q < 5000000; q++) {
        // the midpoint of two adjacent floats (a tie), and one double ulp either side
        const float f = echo::from_bits32((uint32_t)(rng() % 0x7f7fffffu));
        const double lo = (double)f, hi = (double)std::nextafter(f, INFINITY);
        const double mid = 0.5 * (lo + hi);
        check(mid);
        check(std::nextafter(mid, 0.0));
        check(std::nextafter(mid, INFINITY));
        check(-mid);
    }
    const double edge[] = {0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38,
                           3.4028235677973362e38, 1.1754943508222875e-38, 1.1754942106924411e-38,
                           1.401298464324817e-45, 7.006492321624085e-46, INFINITY, -INFINITY,
                           NAN, 1e300, -1e-300};
    for (double x : edge) check(x);
    std::printf("widening %ld checked, %ld mismatches; narrowing %ld checked, %ld mismatches\n",
                n_w, bad_w, n_n, bad_n);
    return (bad_w || bad_n) ? 1 : 0;
}
