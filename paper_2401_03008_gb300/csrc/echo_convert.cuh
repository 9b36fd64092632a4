// Conversions between binary32 and binary64 on the integer pipe.
//
// On GB300 a hardware conversion between float and double (F2F) issues on the
// FP64 pipe, which serves only two thread operations per clock per SM; the mixed
// path converts every reconstructed right-hand side to double and every
// primitive to float, so those conversions would take a sizeable share of the
// scarce pipe.  These functions do the same conversions with integer operations
// on the IEEE-754 bit fields (sign, biased exponent, significand; IEEE 754-2008,
// Sec. 3.4) and give the same results as the hardware conversion:
//  - widening is exact for every input (a NaN keeps its payload and comes out
//    quiet, as the hardware conversion makes it);
//  - narrowing rounds to nearest, ties to even, for results in the normal float
//    range and hands zero, subnormal, overflowing, infinite and NaN inputs to the
//    hardware conversion (rare on this path: a warp takes that branch only if one
//    of its lanes needs it).
// They are host-and-device functions so that the host compiler can check them
// against its own conversions over every class of input.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define ECHO_HD __host__ __device__ __forceinline__
#else
#define ECHO_HD inline
#endif

namespace echo {

ECHO_HD uint32_t bits32(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    return b;
}

ECHO_HD uint64_t bits64(double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}

ECHO_HD float from_bits32(uint32_t b)
{
    float x;
    memcpy(&x, &b, 4);
    return x;
}

ECHO_HD double from_bits64(uint64_t b)
{
    double x;
    memcpy(&x, &b, 8);
    return x;
}

ECHO_HD int clz32(uint32_t m)
{
#ifdef __CUDA_ARCH__
    return __clz((int)m);
#else
    return m ? __builtin_clz(m) : 32;
#endif
}

// float -> double, exact.  Exponent rebias 127 -> 1023 (add 896); a subnormal
// float m 2^-149 becomes the normal double with its leading bit made implicit.
ECHO_HD double to_f64(float x)
{
    const uint32_t b = bits32(x);
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    const uint32_t e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    uint64_t ed, md;
    if (e == 0u) {
        if (m == 0u) return from_bits64(sign);
        const int s = clz32(m) - 8;  // brings the leading bit of m to bit 23
        ed = (uint64_t)(897 - s);
        md = (uint64_t)((m << s) & 0x7fffffu);
    } else {
        ed = e == 0xffu ? 0x7ffull : (uint64_t)(e + 896u);
        md = (e == 0xffu && m) ? (m | 0x400000u) : m;
    }
    return from_bits64(sign | (ed << 52) | (md << 29));
}

ECHO_HD double to_f64(double x) { return x; }

// double -> float, round to nearest even
ECHO_HD float to_f32(double x)
{
    const uint64_t b = bits64(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // float biased exponent
    if (e <= 0 || e >= 255) return (float)x;
    const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 of the 52 bits
    const uint32_t rest = lo & 0x1fffffffu;                  // the 29 dropped bits
    uint32_t r = ((uint32_t)e << 23) | m;
    // a carry out of the significand steps the exponent, up to infinity: as RNE does
    r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return from_bits32((hi & 0x80000000u) | r);
}

ECHO_HD float to_f32(float x) { return x; }

}  // namespace echo
