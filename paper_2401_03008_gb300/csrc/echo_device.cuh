// Device-side building blocks of the ECHO RMHD right-hand side (arXiv 2401.03008).
//
// R is the precision of reconstruction, fluxes and constrained transport: double
// for the FP64 path, float for the mixed path.  The inversion (C2P) and the
// Runge-Kutta accumulation are always double.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "echo_convert.cuh"
#include "echo_mp5dec.cuh"

namespace echo {

// Grid description passed by value to every kernel.
struct Grid {
    int nx, ny, nz;
    long n;            // cells (= faces per direction = edges per direction)
    double h[3];       // cell sizes
    double inv_h[3];
    double hmin;
    double gam;        // adiabatic index
    double gfac;       // gam / (gam - 1)
    double gm1g;       // (gam - 1) / gam
    // FP32 copies of the constants the mixed path's FP32 kernels use (a conversion
    // in the kernel would issue on the FP64 pipe)
    float gm1g32, gam32, gfac32, inv_h32[3];
    // DER weights per direction, divided by h: (75/64, 25/384, 3/640)/h with HO,
    // (1/h, 0, 0) without (set_spacing)
    double derw[3][3];
    float derw32[3][3];
    int ho;            // high-order INT / DER
    int uct;           // 1: staggered field + UCT; 0: cell-centred field, 8-component HLL
    int rec;           // 0: MP5; 1: linear with the MC limiter
    // Owned box [lo, hi) per direction: the cells whose inversion statistics and
    // right-face speeds count (the whole grid, except for a padded subdomain, whose
    // ghost cells are updated too but belong to a neighbour).
    int lo[3], hi[3];
    int primary;       // 1: this grid advances the step counter
};

// Cell sizes and what derives from them (1/h, the DER weights in both precisions,
// the smallest h); ho must be set first.
inline void set_spacing(Grid &g, const double h[3])
{
    for (int d = 0; d < 3; d++) {
        g.h[d] = h[d];
        g.inv_h[d] = 1.0 / h[d];
        g.inv_h32[d] = (float)g.inv_h[d];
        const double w[3] = {g.ho ? 75.0 / 64.0 : 1.0, g.ho ? 25.0 / 384.0 : 0.0,
                             g.ho ? 3.0 / 640.0 : 0.0};
        for (int m = 0; m < 3; m++) {
            g.derw[d][m] = w[m] / h[d];
            g.derw32[d][m] = (float)g.derw[d][m];
        }
    }
    g.hmin = fmin(h[0], fmin(h[1], h[2]));
}

// a grid constant in the precision R (the FP32 copy for float)
template <typename R> __device__ __forceinline__ R gconst(double d, float f);
template <> __device__ __forceinline__ double gconst<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float gconst<float>(double, float f) { return f; }

// the DER weights of direction d in the precision R
template <typename R> __device__ __forceinline__ const R *derw(const Grid &g, int d);
template <> __device__ __forceinline__ const double *derw<double>(const Grid &g, int d)
{
    return g.derw[d];
}
template <> __device__ __forceinline__ const float *derw<float>(const Grid &g, int d)
{
    return g.derw32[d];
}

// a double in the precision R, rounded to nearest (integer pipe for float)
template <typename R> __device__ __forceinline__ R to_r(double x);
template <> __device__ __forceinline__ double to_r<double>(double x) { return x; }
template <> __device__ __forceinline__ float to_r<float>(double x) { return to_f32(x); }

__device__ __forceinline__ bool owned(const Grid &g, int i, int j, int k)
{
    return i >= g.lo[0] && i < g.hi[0] && j >= g.lo[1] && j < g.hi[1] && k >= g.lo[2] &&
           k < g.hi[2];
}


// Device-side scalars of the time loop and the health counters.
struct DevScalars {
    unsigned long long amax_bits;  // running max of a+, a- (non-negative double bits)
    double amax_last;              // amax of the last step
    double dt;                     // dt of the step in progress
    double t;                      // time (advanced when dt is fixed)
    double t_prev;                 // time at the start of the step in progress
    double t_end;
    double cfl;
    unsigned long long it_sum;     // FP64 Newton iterations summed
    unsigned long long it32_sum;   // FP32 pre-iterations summed (mixed path)
    unsigned long long c2p_calls;
    unsigned int it_max;
    unsigned int fails;            // failed inversions
    unsigned int fallbacks;        // rejected learned guesses
    unsigned int rec_fallbacks;    // interface states reset to first order
    int halt;                      // bit 0: inversion failed, bit 1: t_end reached, bit 2: a
                                   // bounded wait of the fused sweep ran out
    int fail_stage;                // stage (1..3) of the first failure, 0 if none
    long fail_step;                // step index of the first failure
    long step;                     // steps completed
};

// Newton parameters.
struct C2PParams {
    double tol;
    int maxit;
    int guess;  // 0 previous W, 1 W0 = U, 2 learned guess array
    int pre32;  // mixed path: FP32 Newton iterations refine the guess first
};

__device__ __forceinline__ int wrapi(int i, int n)
{
    if ((unsigned)i < (unsigned)n) return i;
    if (i < 0 && i + n >= 0) return i + n;
    if (i >= n && i - n < n) return i - n;
    int r = i % n;
    return r < 0 ? r + n : r;
}

// linear index of cell (i,j,k) (already wrapped)
__device__ __forceinline__ long lin(const Grid &g, int i, int j, int k)
{
    return ((long)k * g.ny + j) * g.nx + i;
}

// cell (i,j,k) moved by s along direction D, wrapped
template <int D>
__device__ __forceinline__ long shifted(const Grid &g, int i, int j, int k, int s)
{
    if (D == 0) i = wrapi(i + s, g.nx);
    else if (D == 1) j = wrapi(j + s, g.ny);
    else k = wrapi(k + s, g.nz);
    return lin(g, i, j, k);
}

// 32-bit linear index of the cell s steps from cell c along direction D (iD: the
// cell's coordinate along D), wrapped; the library keeps grids below 2^31 cells
template <int D>
__device__ __forceinline__ int sidx(const Grid &g, int c, int iD, int s)
{
    const int nD = D == 0 ? g.nx : (D == 1 ? g.ny : g.nz);
    const int stride = D == 0 ? 1 : (D == 1 ? g.nx : g.nx * g.ny);
    return c + (wrapi(iD + s, nD) - iD) * stride;
}

__device__ __forceinline__ long shifted_rt(const Grid &g, int i, int j, int k, int d, int s)
{
    if (d == 0) i = wrapi(i + s, g.nx);
    else if (d == 1) j = wrapi(j + s, g.ny);
    else k = wrapi(k + s, g.nz);
    return lin(g, i, j, k);
}

__device__ __forceinline__ void coords(const Grid &g, long c, int &i, int &j, int &k)
{
    // the library limits grids to < 2^31 cells, so 32-bit division suffices
    unsigned cu = (unsigned)c, q = cu / (unsigned)g.nx;
    i = (int)(cu - q * (unsigned)g.nx);
    unsigned kk = q / (unsigned)g.ny;
    k = (int)kk;
    j = (int)(q - kk * (unsigned)g.ny);
}

// ---------------------------------------------------------------------------
// 1-D operators (REC, INT, DER of Sec. 3)
// ---------------------------------------------------------------------------

// Comparisons.  On GB300 the FP64 pipe issues two thread operations per clock per
// SM and a double compare (DSETP) costs as much there as an FMA.  A double maps to
// an ordered 64-bit integer key (the sign-magnitude bits with the magnitude
// flipped for negative values), so compares, min and max of doubles run on the
// integer pipe instead; exact for every non-NaN value (+0 and -0 order as -0 < +0,
// which no result here depends on).  float keeps the native compares.
__device__ __forceinline__ long long okey(double x)
{
    long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool gtz(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool ltz(double x) { return okey(x) < -1; }
__device__ __forceinline__ bool lt(double a, double b) { return okey(a) < okey(b); }
__device__ __forceinline__ bool le(double a, double b) { return okey(a) <= okey(b); }
__device__ __forceinline__ bool finite64(double x)
{
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool gtz(float x) { return x > 0.f; }
__device__ __forceinline__ bool ltz(float x) { return x < 0.f; }
__device__ __forceinline__ bool lt(float a, float b) { return a < b; }
__device__ __forceinline__ bool le(float a, float b) { return a <= b; }

// 4 x, exact.  For a double the biased exponent field is stepped by 2 on the
// integer pipe instead of spending an FP64-pipe multiply; valid for every x whose
// exponent field lies in [1, 2044], i.e. every normal x with |x| < 2^1022.  Any
// other x comes back unchanged: exact for zero, infinity and NaN, off by the factor
// 4 for a subnormal x (|x| < 2.3e-308) and for |x| >= 2^1022, magnitudes that the
// differences compared with the limiter's 1e-10 threshold never reach.
__device__ __forceinline__ double times4(double x)
{
    const long long b = __double_as_longlong(x);
    const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    return e - 1u < 2044u ? __longlong_as_double(b + (2LL << 52)) : x;
}
__device__ __forceinline__ float times4(float x) { return 4.f * x; }

// 1/x and 1/sqrt(x) for the FP64 path with fewer FP64 operations than the library
// forms: an FP32 seed y0 (the hardware approximation of a float copy taken on the
// integer pipe, relative error ~2^-22) and one third-order correction in FP64 --
// Householder's order-3 step, i.e. the series 1/(1 - e) = 1 + e + e^2 + ... with
// e = 1 - x y0 for 1/x, and (1 - e)^(-1/2) = 1 + e/2 + 3 e^2/8 + ... with e = 1 - x y0^2
// for 1/sqrt(x) -- whose truncation error (~e^3 < 2^-64) lies below the FP64 rounding,
// so the results are within about one unit in the last place (tests compare them
// with CUDA's 1.0/x and rsqrt on the GPU).  An x whose
// float copy is zero, infinite or not a number (magnitudes beyond the float range,
// x <= 0 for the square root, NaN) takes the library form.
__device__ __forceinline__ double rcp64(double x)
{
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(trunc_f32(x)));
    if (!(fabsf(yf) < INFINITY && yf != 0.f)) return 1.0 / x;
    const double y0 = to_f64(yf);
    const double e = fma(-x, y0, 1.0);
    return fma(y0, fma(e, e, e), y0);
}
__device__ __forceinline__ double rsqrt64(double x)
{
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(trunc_f32(x)));
    if (!(yf < INFINITY && yf > 0.f)) return rsqrt(x);
    const double y0 = to_f64(yf);
    const double e = fma(-(x * y0), y0, 1.0);
    return fma(y0, e * fma(0.375, e, 0.5), y0);
}
// the precision-generic forms used by the sweeps
__device__ __forceinline__ double rcp_r(double x) { return rcp64(x); }
__device__ __forceinline__ float rcp_r(float x) { return 1.f / x; }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt64(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }

template <typename R> __device__ __forceinline__ R rmin(R a, R b) { return lt(a, b) ? a : b; }
template <typename R> __device__ __forceinline__ R rmax(R a, R b) { return lt(b, a) ? a : b; }

template <typename R>
__device__ __forceinline__ R minmod2(R a, R b)
{
    if (gtz(a) && gtz(b)) return rmin(a, b);
    if (ltz(a) && ltz(b)) return rmax(a, b);
    return R(0);
}

template <typename R>
__device__ __forceinline__ R minmod4(R a, R b, R c, R d)
{
    if (gtz(a) && gtz(b) && gtz(c) && gtz(d)) return rmin(rmin(a, b), rmin(c, d));
    if (ltz(a) && ltz(b) && ltz(c) && ltz(d)) return rmax(rmax(a, b), rmax(c, d));
    return R(0);
}

// MP5 value at i+1/2 from (u_{i-2}, ..., u_{i+2}): fifth-order point-value
// interpolant (3, -20, 90, 60, -5)/128 bounded by the monotonicity-preserving
// limiter of Suresh & Huynh (alpha = 4, eps = 1e-10).  Split in two: the smooth
// candidate with its test, and the limiting that only a few interfaces need.
template <typename R>
__device__ __forceinline__ bool mp5_smooth(R um2, R um1, R u0, R up1, R up2, R dp, R &uor)
{
    // dp = up1 - u0 (the caller shares it between the two states of a face).  The
    // test reads (uor - u0)(uor - ump) <= eps with ump = u0 + minmod(dp, alpha (u0 - um1)),
    // so it needs only d = uor - u0, whose weights are the interpolant's with 1
    // taken from the centre one (90/128 - 1 = -38/128; all exact binary fractions)
    // (alpha = 4: the product alpha (u0 - um1) is times4)
    const R d = R(0.0234375) * um2 - R(0.15625) * um1 - R(0.296875) * u0 + R(0.46875) * up1 -
                R(0.0390625) * up2;
    uor = u0 + d;
    if constexpr (sizeof(R) == 8) {
        // FP64 path: the test in FP32 with its error bound (echo_mp5dec.cuh); FP64
        // only where that cannot decide (about 1e-4 of the tests on the turbulence).
        // up1 - u0 is the caller's dp to the bit (the mirrored state passes -dp).
        const int r = mp5_test32(d, um1, u0, up1);
        if (r >= 0) return r != 0;
        return le(d * (d - minmod2(up1 - u0, times4(u0 - um1))), R(1e-10));
    }
    return le(d * (d - minmod2(dp, times4(u0 - um1))), R(1e-10));
}

template <typename R>
__device__ __forceinline__ bool mp5_smooth(R um2, R um1, R u0, R up1, R up2, R &uor)
{
    return mp5_smooth(um2, um1, u0, up1, up2, up1 - u0, uor);
}

template <typename R>
__device__ __forceinline__ R mp5_limit(R um2, R um1, R u0, R up1, R up2, R uor)
{
    const R alpha = R(4);
    R djm1 = um2 - R(2) * um1 + u0;
    R dj = um1 - R(2) * u0 + up1;
    R djp1 = u0 - R(2) * up1 + up2;
    R dm4p = minmod4(R(4) * dj - djp1, R(4) * djp1 - dj, dj, djp1);
    R dm4m = minmod4(R(4) * dj - djm1, R(4) * djm1 - dj, dj, djm1);
    R uul = u0 + alpha * (u0 - um1);
    R uav = R(0.5) * (u0 + up1);
    R umd = uav - R(0.5) * dm4p;
    R ulc = u0 + R(0.5) * (u0 - um1) + R(4) / R(3) * dm4m;
    R umin = rmax(rmin(rmin(u0, up1), umd), rmin(rmin(u0, uul), ulc));
    R umax = rmin(rmax(rmax(u0, up1), umd), rmax(rmax(u0, uul), ulc));
    return uor + minmod2(umin - uor, umax - uor);
}

template <typename R>
__device__ __forceinline__ R mp5(R um2, R um1, R u0, R up1, R up2)
{
    R uor;
    if (mp5_smooth(um2, um1, u0, up1, up2, uor)) return uor;
    return mp5_limit(um2, um1, u0, up1, up2, uor);
}

// Deferred limiting.  Most interfaces pass the smooth test; the few that do not
// are scattered over most warps, and limiting them in place would run the
// limiter with a handful of lanes active.  Instead a thread queues its five
// stencil values and the candidate in shared memory; after a barrier the whole
// block limits the queued entries with full warps, and each thread collects its
// results.  Same arithmetic as mp5(), so the same results.  Entries beyond QMAX
// are limited in place.
template <typename R, int NSLOT, int QMAX, int NT>
struct Mp5Queue {
    R val[QMAX][6];                    // um2, um1, u0, up1, up2, uor
    R res[QMAX];
    unsigned short slot[NSLOT][NT];    // queue entry of (slot, thread)
    int count;

    __device__ __forceinline__ void reset()
    {
        if (threadIdx.x == 0) count = 0;
    }
    // value of the reconstruction in slot k of this thread (placeholder if queued).
    // The lanes of a warp that need the limiter take consecutive entries with one
    // shared-memory atomic per warp; a warp whose lanes are all smooth skips the
    // queue on a warp-uniform branch.
    __device__ __forceinline__ R defer(R um2, R um1, R u0, R up1, R up2, R dp, int k,
                                       unsigned &mask)
    {
        R uor;
        const bool smooth = mp5_smooth(um2, um1, u0, up1, up2, dp, uor);
        const unsigned am = __activemask();
        const unsigned need = __ballot_sync(am, !smooth);
        if (need == 0u) return uor;
        const int lane = threadIdx.x & 31, leader = __ffs(need) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&count, __popc(need));
        base = __shfl_sync(am, base, leader);
        if (smooth) return uor;
        const int e = base + __popc(need & ((1u << lane) - 1u));
        if (e < QMAX) {
            val[e][0] = um2;
            val[e][1] = um1;
            val[e][2] = u0;
            val[e][3] = up1;
            val[e][4] = up2;
            val[e][5] = uor;
            slot[k][threadIdx.x] = (unsigned short)e;
            mask |= 1u << k;
            return uor;
        }
        return mp5_limit(um2, um1, u0, up1, up2, uor);
    }
    // whole block, between two barriers
    __device__ __forceinline__ void process()
    {
        const int m = count < QMAX ? count : QMAX;
        for (int e = threadIdx.x; e < m; e += NT)
            res[e] = mp5_limit(val[e][0], val[e][1], val[e][2], val[e][3], val[e][4], val[e][5]);
    }
    __device__ __forceinline__ R get(int k) const { return res[slot[k][threadIdx.x]]; }
};

// Linear reconstruction with the monotonized-central slope
// minmod(2 (u_i - u_{i-1}), (u_{i+1} - u_{i-1})/2, 2 (u_{i+1} - u_i)): value at i+1/2
template <typename R>
__device__ __forceinline__ R mc_val(R um1, R u0, R up1)
{
    R a = R(2) * (u0 - um1), b = R(0.5) * (up1 - um1), c = R(2) * (up1 - u0);
    R sl = R(0);
    if (gtz(a) && gtz(b) && gtz(c)) sl = rmin(a, rmin(b, c));
    else if (ltz(a) && ltz(b) && ltz(c)) sl = rmax(a, rmax(b, c));
    return u0 + R(0.5) * sl;
}

// left state at i+1/2 from s[0..5] = u_{i-2..i+3}, and the mirrored right state
template <typename R>
__device__ __forceinline__ void mp5_lr(const R *s, R &L, R &Rr)
{
    L = mp5(s[0], s[1], s[2], s[3], s[4]);
    Rr = mp5(s[5], s[4], s[3], s[2], s[1]);
}

// INT: staggered values at i-3/2, i-1/2, i+1/2, i+3/2 -> centre
template <typename R>
__device__ __forceinline__ R int_c(R a, R b, R c, R d, int ho)
{
    if (ho) return (-a + R(9) * b + R(9) * c - d) * R(0.0625);
    return R(0.5) * (b + c);
}

// cell-centred field at cell c: INT of the staggered components (UCT) or the cell
// values themselves (UCT off)
template <typename BT>
__device__ __forceinline__ BT cell_field_t(const Grid &g, const BT *__restrict__ Bf, long c,
                                           int i, int j, int k, int d)
{
    const BT *b = Bf + d * g.n;
    if (!g.uct) return b[c];
    const int ci = (int)c;
    int sm2, sm1, sp1;
    if (d == 0) {
        sm2 = sidx<0>(g, ci, i, -2);
        sm1 = sidx<0>(g, ci, i, -1);
        sp1 = sidx<0>(g, ci, i, 1);
    } else if (d == 1) {
        sm2 = sidx<1>(g, ci, j, -2);
        sm1 = sidx<1>(g, ci, j, -1);
        sp1 = sidx<1>(g, ci, j, 1);
    } else {
        sm2 = sidx<2>(g, ci, k, -2);
        sm1 = sidx<2>(g, ci, k, -1);
        sp1 = sidx<2>(g, ci, k, 1);
    }
    return int_c(b[sm2], b[sm1], b[c], b[sp1], g.ho);
}

template <typename BT>
__device__ __forceinline__ double cell_field(const Grid &g, const BT *__restrict__ Bf, long c,
                                             int i, int j, int k, int d)
{
    return to_f64(cell_field_t(g, Bf, c, i, j, k, d));
}

// DER: derivative at a centre from staggered values s[0..5] at i-5/2..i+5/2.
// High order corrects each staggered value by -d2/24 + 3 d4/640 before the
// difference; expanded, the two corrected values combine into the single stencil
// (75/64 (s3-s2) - 25/384 (s4-s1) + 3/640 (s5-s0)) / h, used here (no divisions).
template <typename R>
__device__ __forceinline__ R der_c(const R *s, R inv_h, int ho)
{
    if (!ho) return (s[3] - s[2]) * inv_h;
    const R c0 = R(75.0 / 64.0), c1 = R(25.0 / 384.0), c2 = R(3.0 / 640.0);
    return (c0 * (s[3] - s[2]) - c1 * (s[4] - s[1]) + c2 * (s[5] - s[0])) * inv_h;
}

// acc - DER(s) and acc + DER(s) with the direction's weights w divided by h
// (Grid::derw): the same stencil as der_c, each term one fused multiply-add.
template <typename R>
__device__ __forceinline__ R der_sub(R acc, const R *s, const R *w, int ho)
{
    acc = acc - w[0] * (s[3] - s[2]);
    if (!ho) return acc;
    acc = acc + w[1] * (s[4] - s[1]);
    return acc - w[2] * (s[5] - s[0]);
}

template <typename R>
__device__ __forceinline__ R der_add(R acc, const R *s, const R *w, int ho)
{
    acc = acc + w[0] * (s[3] - s[2]);
    if (!ho) return acc;
    acc = acc - w[1] * (s[4] - s[1]);
    return acc + w[2] * (s[5] - s[0]);
}

// ---------------------------------------------------------------------------
// Point-wise physics (Sec. 2, flat space, ideal MHD, ideal gas)
// ---------------------------------------------------------------------------

// Conserved variables (D, S, U) and field, physical flux along D of all 8, and the
// fast speeds lm <= lp along D, sharing the intermediate quantities.
// s = (rho, vx, vy, vz, p, Bx, By, Bz); v2 = vx^2 + vy^2 + vz^2 (the caller has it).
template <typename R, int D>
__device__ __forceinline__ void phys(const R *s, R v2, R gam, R gfac, R *U, R *F, R &lm, R &lp)
{
    const R rho = s[0], vx = s[1], vy = s[2], vz = s[3], pg = s[4];
    const R bx = s[5], by = s[6], bz = s[7];
    R omv2 = R(1) - v2;
    R lor = rsqrt_r(omv2);
    R lor2 = lor * lor;
    R rhoh = rho + gfac * pg;
    R w = rhoh * lor2;
    // E = -v x B
    R ex = -(vy * bz - vz * by);
    R ey = -(vz * bx - vx * bz);
    R ez = -(vx * by - vy * bx);
    R b2 = bx * bx + by * by + bz * bz;
    R vb = vx * bx + vy * by + vz * bz;
    // |v x B|^2 = v^2 B^2 - (v.B)^2 and E x B = B^2 v - (v.B) B (Lagrange and
    // triple-product identities): fewer operations than from the components
    R e2 = v2 * b2 - vb * vb;
    R D0 = rho * lor;
    R wb = w + b2;
    R Sx = wb * vx - vb * bx;
    R Sy = wb * vy - vb * by;
    R Sz = wb * vz - vb * bz;
    R ptot = pg + R(0.5) * (e2 + b2);
    U[0] = D0;
    U[1] = Sx;
    U[2] = Sy;
    U[3] = Sz;
    U[4] = w - pg + R(0.5) * (e2 + b2);
    U[5] = bx;
    U[6] = by;
    U[7] = bz;
    const R vd = s[1 + D];
    const R Ed = D == 0 ? ex : (D == 1 ? ey : ez);
    const R Bd = s[5 + D];
    const R wvd = w * vd;
    F[0] = D0 * vd;
    F[1] = wvd * vx - ex * Ed - bx * Bd + (D == 0 ? ptot : R(0));
    F[2] = wvd * vy - ey * Ed - by * Bd + (D == 1 ? ptot : R(0));
    F[3] = wvd * vz - ez * Ed - bz * Bd + (D == 2 ? ptot : R(0));
    F[4] = D == 0 ? Sx : (D == 1 ? Sy : Sz);
    F[5] = vd * bx - vx * Bd;
    F[6] = vd * by - vy * Bd;
    F[7] = vd * bz - vz * Bd;
    // Approximate fast magnetosonic speeds
    //   lambda = [v_d (1 - w2) +- sqrt(w2 (1 - v^2) ((1 - v^2 w2) - v_d^2 (1 - w2)))] / (1 - v^2 w2)
    // with cs2 = gam p / rho h, ca2 = b^2 / (rho h + b^2), w2 = cs2 + ca2 - cs2 ca2.
    // Since 1 - w2 = (1 - cs2)(1 - ca2) = P / den and w2 = Q / den with
    // P = rho h - gam p, Q = b^2 + gam p, den = rho h + b^2, multiplying through by den
    // leaves lambda = [v_d P +- sqrt((1 - v^2) Q K)] / Y, Y = den - v^2 Q,
    // K = Y - v_d^2 P: no reciprocal of rho h or den at all.
    R bb2 = b2 * omv2 + vb * vb;
    R gp = gam * pg;
    R P = rhoh - gp;
    R Q = bb2 + gp;
    R Y = (rhoh + bb2) - v2 * Q;
    R K = Y - vd * vd * P;
    R disc = omv2 * Q * K;
    // sqrt(disc)/Y and 1/Y from one reciprocal square root q = 1/sqrt(disc Y^2):
    // sqrt(disc)/Y = disc q and 1/Y = Y disc q^2 (disc > 0); disc <= 0 takes 1/Y
    const R a = vd * P;
    if (gtz(disc)) {
        R q = rsqrt_r(disc * Y * Y);
        R srx = disc * q;
        R inv = Y * srx * q;
        lp = a * inv + srx;
        lm = a * inv - srx;
    } else {
        lp = lm = a / Y;
    }
}

// ---------------------------------------------------------------------------
// UCT four-state edge field; (a, b, c) cyclic, edge along c at (a+1/2, b+1/2).
// va/vb[s][t]: velocity components a and b of the a-face state s (L/R) reconstructed
// along b to side t; Ba[t]: B_a along b; Bb[s]: B_b along a.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R uct_point(const R va[2][2], const R vb[2][2], const R Ba[2],
                                       const R Bb[2], R apa, R ama, R apb, R amb)
{
    R sa = apa + ama, sb = apb + amb;
    R e4 = R(0);
    R isa = R(0), isb = R(0);
    const bool pa = gtz(sa), pb = gtz(sb);
    if (pa && pb) {
        R wa[2] = {apa, ama}, wb[2] = {apb, amb};
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int t = 0; t < 2; t++)
                e4 += wa[s] * wb[t] * (vb[s][t] * Ba[t] - va[s][t] * Bb[s]);
        R r = rcp_r(sa * sb);
        e4 = e4 * r;
        isa = sb * r;
        isb = sa * r;
    } else {
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int t = 0; t < 2; t++)
                e4 += R(0.25) * (vb[s][t] * Ba[t] - va[s][t] * Bb[s]);
    }
    if (pa && !pb) isa = rcp_r(sa);
    if (pb && !pa) isb = rcp_r(sb);
    R da = apa * ama * (Bb[1] - Bb[0]) * isa;
    R db = apb * amb * (Ba[1] - Ba[0]) * isb;
    return e4 + da - db;
}

// ---------------------------------------------------------------------------
// C2P: Newton on W = rho h G^2 (always double)
// ---------------------------------------------------------------------------
struct C2PInv {
    double D, S2, B2, SB, U, gm1g;
    float gm1g32;
};

// v^2(W) and r = 1/(W (W + B^2)); valid when W > 0, finite and v^2 < 1
__device__ __forceinline__ bool c2p_eval(const C2PInv &q, double W, double &v2, double &r)
{
    if (!gtz(W) || !finite64(W)) return false;
    double wb = W + q.B2;
    r = rcp64(W * wb);
    v2 = (q.S2 * W * W + q.SB * q.SB * (q.B2 + 2.0 * W)) * (r * r);
    return finite64(v2) && lt(v2, 1.0);
}

__device__ __forceinline__ bool c2p_ok(const C2PInv &q, double W)
{
    double v2, r;
    return c2p_eval(q, W, v2, r);
}

// FP32 Newton iterations on the same f(W), used by the mixed path to refine the
// starting guess before the FP64 iteration (FP32 issues 64x faster than FP64 on
// GB300).  Stops once a step is below 4e-6 W (FP32 cannot resolve much further);
// returns the refined guess, or W0 unchanged if an iterate leaves the domain or
// is not finite.  The FP64 iteration that follows decides the result.
__device__ __forceinline__ double c2p_pre32(const C2PInv &q, double W0, int &iters, float &idf)
{
    const float D = to_f32(q.D), S2 = to_f32(q.S2), B2 = to_f32(q.B2), SB = to_f32(q.SB);
    const float U = to_f32(q.U), gm1g = q.gm1g32, SB2 = SB * SB;
    float W = to_f32(W0);
    iters = 0;
    idf = 0.f;
    if (!(W > 0.f) || !isfinite(W)) return W0;
    for (int k = 0; k < 8; k++) {
        float wb = W + B2;
        float r = 1.f / (W * wb);
        float iW = wb * r, iwb = W * r;
        float v2 = (S2 * W * W + SB2 * (B2 + 2.f * W)) * (r * r);
        if (!(v2 < 1.f) || !isfinite(v2)) return W0;
        float omv2 = 1.f - v2;
        float isq = rsqrtf(omv2);
        float sq1 = omv2 * isq;
        float iW2 = iW * iW;
        float p = gm1g * (W * omv2 - D * sq1);
        float dv2 = -2.f * SB2 * (iW2 * iW) * iwb - 2.f * v2 * iwb;
        float dp = gm1g * (omv2 - W * dv2 + 0.5f * D * dv2 * isq);
        float f = W - p + 0.5f * (1.f + v2) * B2 - 0.5f * SB2 * iW2 - U;
        float df = 1.f - dp + 0.5f * B2 * dv2 + SB2 * (iW2 * iW);
        float rdf = 1.f / df;
        float dW = -f * rdf;
        float Wn = W + dW;
        iters++;
        if (!(Wn > 0.f) || !isfinite(Wn) || !isfinite(rdf)) {
            idf = 0.f;
            return W0;
        }
        W = Wn;
        idf = rdf;
        if (fabsf(dW) <= 4e-6f * W) break;
    }
    return to_f64(W);
}

// Newton on f(W) = W - p(W) + (1 + v^2) B^2/2 - (S.B)^2/(2 W^2) - U with the
// analytic derivative; a trial point outside the domain halves the step; stop
// after an undamped step with |dW| <= tol W and one more polishing step (the chord
// iteration of the mixed path stops after that step).  The domain check of a trial
// point computes v^2 and 1/(W (W+B^2)) there, and the next iteration reuses both,
// so an iteration costs two divisions and one reciprocal square root.
// Returns true on success.  prim = (rho, vx, vy, vz, p); B the cell-centred field.
// the invariants D, S^2, B^2, S.B, U of a cell's conserved state and field
__device__ __forceinline__ C2PInv c2p_invariants(const double *u, const double *B, double gm1g,
                                                 float gm1g32)
{
    C2PInv q;
    q.D = u[0];
    q.S2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    q.B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    q.SB = u[1] * B[0] + u[2] * B[1] + u[3] * B[2];
    q.U = u[4];
    q.gm1g = gm1g;  // (gam - 1)/gam, formed once on the host
    q.gm1g32 = gm1g32;
    return q;
}

// Wfb: a second starting point, taken when W0 lies outside the domain (the
// previous W when W0 is the learned guess; *fb reports that it was taken); pass
// fb = nullptr for none.  MIXED: compile the mixed path's FP32 pre-iterations and
// chord steps (taken when pre32 != 0); the FP64 path's kernels leave them out.
template <bool MIXED>
__device__ __forceinline__ bool c2p_newton(const C2PInv &q, const double *u, const double *B,
                                           double W0, double tol, int maxit, double *prim,
                                           double &Wout, int &iters, int pre32, int &iters32,
                                           double Wfb = 0.0, bool *fb = nullptr)
{
    const double SB2 = q.SB * q.SB;
    iters32 = 0;
    // mixed path: FP32 iterations first; their last derivative then serves every
    // FP64 step (a chord iteration: FP64 residual, FP32-accurate slope, contraction
    // by about the slope's relative error per step), so an FP64 step evaluates f only
    float idf32 = 0.f;
    if (MIXED && pre32) W0 = c2p_pre32(q, W0, iters32, idf32);
    const bool chord = MIXED && idf32 != 0.f;
    const double idf = to_f64(idf32);
    double W = W0, v2 = 0.0, r = 0.0;
    bool ok = c2p_eval(q, W, v2, r);
    if (fb) {
        *fb = !ok;
        if (!ok) {
            W = Wfb;
            ok = c2p_eval(q, W, v2, r);
        }
    }
    for (int k = 0; k < 64 && !ok; k++) {
        W = (gtz(W) && finite64(W)) ? 2.0 * W : fabs(q.U) + 1.0;
        ok = c2p_eval(q, W, v2, r);
    }
    int it = 0;
    bool conv = false, polish = false, have_sq1 = false;
    double sq1f = 0.0;
    while (ok && it < maxit) {
        double wb = W + q.B2;
        double iW = wb * r, iwb = W * r;
        double omv2 = 1.0 - v2;
        double isq = rsqrt64(omv2);
        double sq1 = omv2 * isq;
        double iW2 = iW * iW;
        double p = q.gm1g * (W * omv2 - q.D * sq1);
        double f = W - p + 0.5 * (1.0 + v2) * q.B2 - 0.5 * SB2 * iW2 - q.U;
        double dW, dv2 = 0.0;
        if (!chord) dv2 = -2.0 * SB2 * (iW2 * iW) * iwb - 2.0 * v2 * iwb;
        if (chord) {
            dW = -f * idf;
        } else {
            double dp = q.gm1g * (omv2 - W * dv2 + 0.5 * q.D * dv2 * isq);
            double df = 1.0 - dp + 0.5 * q.B2 * dv2 + SB2 * (iW2 * iW);
            dW = -f * rcp64(df);
        }
        if (!finite64(dW)) break;
        double lam = 1.0, Wn = W + dW, v2n, rn;
        // Mixed path: the chord step that meets the stopping test moves W by at most
        // tol W, so v^2, 1/(W (W + B^2)) and sqrt(1 - v^2) at the new point follow from
        // their values and derivatives at W to second order in dW/W (below 1e-12
        // relative, under the 1e-11 W error the chord stop leaves), in place of one
        // more division and a square root.  A point that this leaves outside the
        // domain takes the exact evaluation below.  (Newton's polishing step keeps the
        // exact evaluation: its lanes reach it at different iterations, and a warp
        // would run both forms.)
        const bool last = chord && le(fabs(Wn - W), tol * Wn);
        if (last) {
            dv2 = -2.0 * SB2 * (iW2 * iW) * iwb - 2.0 * v2 * iwb;
            v2n = v2 + dv2 * dW;
            rn = r - (2.0 * W + q.B2) * (r * r) * dW;
            if (gtz(Wn) && finite64(Wn) && finite64(v2n) && lt(v2n, 1.0) && gtz(rn)) {
                it++;
                sq1f = sq1 - 0.5 * isq * (v2n - v2);
                have_sq1 = true;
                W = Wn;
                v2 = v2n;
                r = rn;
                conv = true;
                break;
            }
        }
        bool okn = c2p_eval(q, Wn, v2n, rn);
        for (int k = 0; k < 60 && !okn; k++) {
            lam *= 0.5;
            Wn = W + lam * dW;
            okn = c2p_eval(q, Wn, v2n, rn);
        }
        it++;
        if (!okn) {
            ok = false;
            break;
        }
        double step = fabs(Wn - W);
        W = Wn;
        v2 = v2n;
        r = rn;
        if (polish) {
            conv = true;
            break;
        }
        if (lam == 1.0 && le(step, tol * W)) {
            // A chord step contracts the error by the slope's relative error
            // (<= ~1e-5 for an FP32-refined slope), so the error left after an undamped
            // step of at most tol W is below 1e-5 tol W: the mixed path stops there,
            // four orders of magnitude under the FP32 rounding of its sweeps.  Newton
            // (FP64 path) takes the polishing step down to the rounding floor.
            if (chord) {
                conv = true;
                break;
            }
            polish = true;
        }
    }
    iters = it;
    Wout = W;
    if (!ok) v2 = fmin(fmax(v2, 0.0), 1.0);
    double omv2 = 1.0 - v2;
    // sqrt(1 - v^2) as (1 - v^2)/sqrt(1 - v^2); a clamped v^2 = 1 (failed cell) gives 0
    double sq1 = have_sq1 ? sq1f : omv2 * rsqrt64(rmax(omv2, 1e-300));
    double p = q.gm1g * (W * omv2 - q.D * sq1);
    double rho = q.D * sq1;
    double wb = W + q.B2;
    double iW = wb * r, iwb = W * r;
    for (int i = 0; i < 3; i++) prim[1 + i] = (u[1 + i] + q.SB * B[i] * iW) * iwb;
    prim[0] = rho;
    prim[4] = p;
    return ok && conv && finite64(p) && finite64(rho) && gtz(p) && gtz(rho) && lt(v2, 1.0);
}

__device__ __forceinline__ bool c2p_newton(const double *u, const double *B, double gm1g,
                                           float gm1g32, double W0, double tol, int maxit,
                                           double *prim, double &Wout, int &iters, int pre32,
                                           int &iters32)
{
    const C2PInv q = c2p_invariants(u, B, gm1g, gm1g32);
    return pre32 ? c2p_newton<true>(q, u, B, W0, tol, maxit, prim, Wout, iters, pre32, iters32)
                 : c2p_newton<false>(q, u, B, W0, tol, maxit, prim, Wout, iters, pre32, iters32);
}

// ---------------------------------------------------------------------------
// warp / block reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_max_r(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// maximum of non-negative doubles through their ordered integer keys (integer pipe)
__device__ __forceinline__ double warp_max_r(double v)
{
    long long k = __double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long q = __shfl_xor_sync(0xffffffffu, k, o);
        k = q > k ? q : k;
    }
    return __longlong_as_double(k);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace echo
