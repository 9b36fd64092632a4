// The MP5 smooth test of the FP64 path decided in FP32 where the decision is certain.
//
// MP5 (Sec. 3 step 2; Suresh & Huynh's limiter) keeps the fifth-order candidate
// u_or = u0 + d where t = d (d - minmod(u_{+1} - u0, 4 (u0 - u_{-1}))) <= 1e-10.  On
// GB300 the FP64 pipe serves two thread operations per clock per SM and bounds the
// FP64 sweeps, while the FP32 pipe and the integer pipe sit mostly idle.  Here t is
// formed in FP32 from float copies of d, u_{-1}, u0, u_{+1} (taken on the integer
// pipe), together with a bound B on its distance from the exact value; when
// t32 + B lies below 1e-10 the candidate is certainly kept, when t32 - B lies above
// it certainly goes to the limiter, and only in between does the caller evaluate
// the test in FP64.  The decision is therefore always the FP64 one.
//
// The bound: each float copy is the double truncated to 24 significant bits
// (relative error below 2^-23; magnitudes under 2^-126 become zero, an absolute
// error below 1.2e-38); each FP32 operation adds at most 2^-24 relative.  With
// U = 2^-22 (twice the truncation unit),
//   |b - b_x|   <= U (|a0| + |a1| + |b|)           b  = a0 - a1
//   |dp - dp_x| <= U (|ap| + |a0| + |dp|)          dp = ap - a0
//   |mm - mm_x| <= max(err dp, 4 err b)            (minmod is 1-Lipschitz in each argument)
//   |d32 - d|   <= U |d32|
//   |e - e_x|   <= err d + err mm + U |e|          e  = d32 - mm
//   |t - t_x|   <= |d32| err e + |e| err d + U |t| (+ second-order terms)
// and B is 1.25 times the last line plus 1e-30 for the flushed magnitudes and the
// rounding of B itself.  Host and device compile the same source (tests check it
// against the FP64 test on random and constructed inputs).
#pragma once

#include "echo_convert.cuh"

#ifndef __CUDACC__
#include <cmath>
#endif

namespace echo {

// a double as a float on the integer pipe, truncated toward zero: relative error
// below 2^-23; magnitudes below 2^-126 give a signed zero, magnitudes beyond the
// float range an infinity, NaN a NaN
ECHO_HD float trunc_f32(double x)
{
    const uint64_t b = bits64(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
    uint32_t r = sign | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    if (e <= 896u) r = sign;
    if (e >= 1151u) {
        const bool nan = e == 0x7ffu && ((hi & 0xfffffu) | lo) != 0u;
        r = sign | 0x7f800000u | (nan ? 0x400000u : 0u);
    }
    return from_bits32(r);
}

ECHO_HD float mp5dec_abs(float x) { return x < 0.f ? -x : x; }

// minmod of two floats (0 unless both have the same sign)
ECHO_HD float mp5dec_minmod(float a, float b)
{
    if (a > 0.f && b > 0.f) return a < b ? a : b;
    if (a < 0.f && b < 0.f) return a > b ? a : b;
    return 0.f;
}

// 1: t <= 1e-10 certainly (keep the candidate); 0: t > 1e-10 certainly (limit);
// -1: undecided in FP32 (the caller evaluates t in FP64).  d = u_or - u0.
ECHO_HD int mp5_test32(double d, double um1, double u0, double up1)
{
    const float a1 = trunc_f32(um1), a0 = trunc_f32(u0), ap = trunc_f32(up1);
    const float d32 = trunc_f32(d);
    const float b = a0 - a1, dp = ap - a0;
    const float mm = mp5dec_minmod(dp, 4.f * b);
    const float e = d32 - mm;
    const float t = d32 * e;
    const float U = 2.384185791015625e-7f;  // 2^-22
    const float eb = U * (mp5dec_abs(a0) + mp5dec_abs(a1) + mp5dec_abs(b));
    const float edp = U * (mp5dec_abs(ap) + mp5dec_abs(a0) + mp5dec_abs(dp));
    const float emm = edp > 4.f * eb ? edp : 4.f * eb;
    const float ed = U * mp5dec_abs(d32);
    const float ee = ed + emm + U * mp5dec_abs(e);
    const float B = 1.25f * (mp5dec_abs(d32) * ee + mp5dec_abs(e) * ed + U * mp5dec_abs(t)) +
                    1e-30f;
    // thresholds on either side of the double 1e-10 with a margin far above the
    // rounding of t + B and t - B
    if (t + B < 0.9999e-10f) return 1;
    if (t - B > 1.0001e-10f) return 0;
    return -1;
}

}  // namespace echo
