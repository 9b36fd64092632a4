// Fused sweep of the mixed path along y or z (Sec. 3, substep steps 2-3 for one
// direction): MP5 reconstruction, physical fluxes, fast speeds, HLL and the DER of
// the fluxes into the right-hand side, in one kernel, the face fluxes never
// leaving the chip.
//
// A block of 128 threads owns a 32 x 4 block of columns along the sweep direction D
// (32 consecutive x, 4 consecutive cells of the third direction) and marches along
// D over a segment of T cells.  Face f (between cells f and f+1 along D) needs the
// primitives of cells f-2..f+3; the block keeps an 8-slot ring of planes (all 8
// primitives of its 128 columns at one coordinate along D, 4 KB each) in shared
// memory, filled by TMA (cp.async.bulk.tensor of a 4-D box of the primitive array,
// this GPU's own memory, no multicast) two steps ahead of their first use, one
// mbarrier per slot.  Each thread keeps the fluxes of the last six faces of its own
// column in registers, so the DER of cell f-2 (faces f-5..f, the high-order stencil)
// follows face f without any exchange.  The deferred MP5 limiting runs per warp
// (queue in shared memory, __syncwarp only); one block barrier per step, after the
// wait for the step's plane, frees the slot that the next TMA (three planes ahead)
// overwrites.  A segment recomputes the 5 faces of its halo (T + 5 faces for T
// cells).
//
// Every wait on an mbarrier is bounded: past the limit the block raises bit 2 of
// the halt flag (the step is then reported as failed and rolled back); its issuing
// thread waits, again bounded, for the block's copies in flight, and it returns.
// The decision is block-uniform (__syncthreads_or).
#pragma once

#include <cuda.h>

#include "echo_internal.h"

namespace echo {

constexpr int SW_COLS = 128;               // columns (threads) of a block: 32 x 4
constexpr int SW_RING = 8;                 // planes in the ring
constexpr int SW_SLOT = 8 * SW_COLS;       // floats of one plane (8 primitives)
constexpr int SW_QW = 64;                  // deferred-limiting entries per warp
constexpr unsigned SW_SPIN = 1u << 22;     // bound of one mbarrier wait (polls)

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// true once the phase with the given parity has completed
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false if the limit was reached
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    for (unsigned k = 0; k < SW_SPIN; k++)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// one plane (all 8 primitives of the block's columns) into a ring slot
__device__ __forceinline__ void tma_plane(float *dst, const CUtensorMap *tm, int c0, int c1,
                                          int c2, unsigned long long *bar)
{
    mbar_expect_tx(bar, SW_SLOT * 4);
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)tm), "r"(c0), "r"(c1), "r"(c2), "r"(0), "r"(smem_u32(bar))
        : "memory");
}

// Deferred MP5 limiting of one warp (the block-wide Mp5Queue's arithmetic, with the
// queue local to the warp): the entry count is a warp-uniform register, so only
// __syncwarp orders the queue's shared memory.
template <int NSLOT>
struct Mp5WarpQueue {
    float val[SW_QW][6];
    float res[SW_QW];
    unsigned char slot[NSLOT][32];

    __device__ __forceinline__ float defer(float um2, float um1, float u0, float up1, float up2,
                                           float dp, int k, unsigned &mask, int lane, int &cnt)
    {
        float uor;
        const bool smooth = mp5_smooth(um2, um1, u0, up1, up2, dp, uor);
        const unsigned need = __ballot_sync(0xffffffffu, !smooth);
        if (need == 0u) return uor;
        const int e = cnt + __popc(need & ((1u << lane) - 1u));
        cnt += __popc(need);
        if (smooth) return uor;
        if (e < SW_QW) {
            val[e][0] = um2;
            val[e][1] = um1;
            val[e][2] = u0;
            val[e][3] = up1;
            val[e][4] = up2;
            val[e][5] = uor;
            slot[k][lane] = (unsigned char)e;
            mask |= 1u << k;
            return uor;
        }
        return mp5_limit(um2, um1, u0, up1, up2, uor);
    }
    __device__ __forceinline__ void process(int lane, int cnt)
    {
        const int m = cnt < SW_QW ? cnt : SW_QW;
        for (int e = lane; e < m; e += 32)
            res[e] = mp5_limit(val[e][0], val[e][1], val[e][2], val[e][3], val[e][4], val[e][5]);
    }
    __device__ __forceinline__ float get(int k, int lane) const { return res[slot[k][lane]]; }
};

// D = 1 (y) or 2 (z).  tm: the primitive array [8][nz][ny][nx] (float) as a 4-D
// tensor (x, y, z, var) with box (32, 4, 1, 8) for D = 2 and (32, 1, 4, 8) for D = 1.
// Columns: x = 32 bx + lane-in-row, o = 4 bo + row (o = y for D = 2, z for D = 1).
// Segment sg covers cells [T sg, T sg + T) along D.  rhs: the cell right-hand side,
// holding the x sweep's contribution (this kernel subtracts its DER).
template <int D>
__global__ void __launch_bounds__(SW_COLS, 5)
k_sweep(Grid g, const __grid_constant__ CUtensorMap tm, const float *__restrict__ prim,
        const float *__restrict__ Bf, float *__restrict__ rhs, float *__restrict__ fd,
        DevScalars *sc, int T, int want_amax)
{
    static_assert(D == 1 || D == 2, "the x sweep keeps the separate flux and DER kernels");
    constexpr int E1 = (D + 1) % 3;
    __shared__ __align__(128) float ring[SW_RING][SW_SLOT];
    __shared__ __align__(8) unsigned long long bars[SW_RING];
    __shared__ Mp5WarpQueue<14> wq[SW_COLS / 32];
    __shared__ float red[SW_COLS / 32];
    __shared__ int halted;
    // the flag may be raised by another block of this launch: read it once, so that
    // the whole block leaves or stays (the march has block barriers)
    if (threadIdx.x == 0) halted = *(volatile int *)&sc->halt;
    __syncthreads();
    if (halted) return;
    const int nD = D == 1 ? g.ny : g.nz;
    const int nO = D == 1 ? g.nz : g.ny;  // the third direction
    const long n = g.n;
    const long strideD = D == 1 ? (long)g.nx : (long)g.nx * g.ny;
    const long strideO = D == 1 ? (long)g.nx * g.ny : (long)g.nx;
    const int nbx = (g.nx + 31) >> 5, nbo = (nO + 3) >> 2;
    unsigned b = blockIdx.x;
    const int bx = (int)(b % nbx);
    b /= nbx;
    const int bo = (int)(b % nbo);
    const int sg = (int)(b / nbo);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x = 32 * bx + lane, o = 4 * bo + warp;
    const bool active = x < g.nx && o < nO;
    const long cbase = (long)o * strideO + x;  // the column's cell at coordinate 0 along D
    const int k0 = T * sg;
    const int kend = min(k0 + T, nD);          // cells [k0, kend) of this segment
    const int p0 = k0 - 5;                     // first plane of the ring
    const int nplanes = (kend - k0) + 10;
    const int cx = 32 * bx, co = 4 * bo;
    auto wrapD = [&](int p) { p %= nD; return p < 0 ? p + nD : p; };
    auto issue = [&](int lp) {  // plane p0 + lp into slot lp % 8
        const int p = wrapD(p0 + lp), s = lp & (SW_RING - 1);
        if (D == 2) tma_plane(ring[s], &tm, cx, co, p, &bars[s]);
        else tma_plane(ring[s], &tm, cx, p, co, &bars[s]);
    };
    if (tid == 0) {
        for (int s = 0; s < SW_RING; s++) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int lp = 0; lp < SW_RING && lp < nplanes; lp++) issue(lp);
    }
    __syncthreads();
    Mp5WarpQueue<14> &q = wq[warp];
    const float gam = g.gam32, gfac = g.gfac32, *w = g.derw32[D];
    float Fh[6][5];  // fluxes of faces f-5..f of this column
    float amax = 0.f;
    unsigned nfb = 0;
    int issued = SW_RING - 1;  // last ring plane requested (thread 0)
    // the first face reads planes 0..5: each thread waits for 0..4 here and for the
    // plane that completes a face's stencil in the loop (the copies land in any order)
    bool ok0 = true;
    for (int lq = 0; lq < 5; lq++) ok0 &= mbar_wait(&bars[lq], 0u);
    for (int f = k0 - 3; f <= kend + 1; f++) {
        // global loads that do not depend on the planes go first, so that their latency
        // overlaps the wait and the reconstruction: the normal field of face f and the
        // right-hand side of cell f - 2, whose DER follows this face
        const long fc = cbase + (long)wrapD(f) * strideD;  // face f belongs to cell f
        const float bn = active ? Bf[D * n + fc] : 0.f;
        const int kc = f - 2;
        const bool derc = active && kc >= k0 && kc < kend;
        const long cc = cbase + (long)kc * strideD;
        float rh[5];
#pragma unroll
        for (int qq = 0; qq < 5; qq++) rh[qq] = derc ? rhs[qq * n + cc] : 0.f;
        const int lp = f + 3 - p0;  // the plane f + 3 completes the stencil of face f
        const bool ok = mbar_wait(&bars[lp & (SW_RING - 1)], (unsigned)(lp >> 3) & 1u) && ok0;
        // every thread is past face f - 1 here, so plane f - 3's slot is free
        if (__syncthreads_or(!ok)) {
            // a copy did not arrive: report, let this block's copies in flight land
            // (bounded), leave
            if (tid == 0) {
                // stage 1 (the step's first, which asks for the speed maximum) or a later
                // one: the host restores the step's start state for the latter
                if (atomicCAS(&sc->fail_stage, 0, want_amax ? 1 : 2) == 0)
                    sc->fail_step = (long)sc->step;
                atomicOr(&sc->halt, 4);
                for (int lq = lp; lq <= issued; lq++)
                    mbar_wait(&bars[lq & (SW_RING - 1)], (unsigned)(lq >> 3) & 1u);
            }
            return;
        }
        if (tid == 0 && lp + 2 < nplanes && lp + 2 > issued) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(lp + 2);  // plane f + 5 into the slot of plane f - 3
            issued = lp + 2;
        }
        // MP5 left/right states of the 7 reconstructed primitives at face f
        const float *pl[6];
#pragma unroll
        for (int m = 0; m < 6; m++) pl[m] = ring[(f - 2 + m - p0) & (SW_RING - 1)];
        float L[8], R[8];
        unsigned mask = 0;
        int cnt = 0;
#pragma unroll
        for (int v = 0; v < 8; v++) {
            if (v == 5 + D) continue;
            float s[6];
#pragma unroll
            for (int m = 0; m < 6; m++) s[m] = pl[m][v * SW_COLS + tid];
            const float dc = s[3] - s[2];
            L[v] = q.defer(s[0], s[1], s[2], s[3], s[4], dc, 2 * v - (v > 5 + D ? 2 : 0), mask,
                           lane, cnt);
            R[v] = q.defer(s[5], s[4], s[3], s[2], s[1], -dc, 2 * v + 1 - (v > 5 + D ? 2 : 0),
                           mask, lane, cnt);
        }
        __syncwarp();
        q.process(lane, cnt);
        __syncwarp();
#pragma unroll
        for (int v = 0; v < 8; v++) {
            if (v == 5 + D) continue;
            const int kl = 2 * v - (v > 5 + D ? 2 : 0);
            if (mask & (1u << kl)) L[v] = q.get(kl, lane);
            if (mask & (1u << (kl + 1))) R[v] = q.get(kl + 1, lane);
        }
        L[5 + D] = bn;
        R[5 + D] = bn;
        // positivity: a state with rho <= 0, p <= 0 or v^2 >= 1 takes the cell value
        float v2L = L[1] * L[1] + L[2] * L[2] + L[3] * L[3];
        float v2R = R[1] * R[1] + R[2] * R[2] + R[3] * R[3];
        if (!(L[0] > 0.f) || !(L[4] > 0.f) || !(v2L < 1.f)) {
#pragma unroll
            for (int v = 0; v < 8; v++)
                if (v != 5 + D) L[v] = pl[2][v * SW_COLS + tid];
            v2L = L[1] * L[1] + L[2] * L[2] + L[3] * L[3];
            nfb++;
        }
        if (!(R[0] > 0.f) || !(R[4] > 0.f) || !(v2R < 1.f)) {
#pragma unroll
            for (int v = 0; v < 8; v++)
                if (v != 5 + D) R[v] = pl[3][v * SW_COLS + tid];
            v2R = R[1] * R[1] + R[2] * R[2] + R[3] * R[3];
            nfb++;
        }
        float UL[8], FL[8], UR[8], FR[8], lmL, lpL, lmR, lpR;
        phys<float, D>(L, v2L, gam, gfac, UL, FL, lmL, lpL);
        phys<float, D>(R, v2R, gam, gfac, UR, FR, lmR, lpR);
        const float ap = fmaxf(0.f, fmaxf(lpL, lpR));
        const float am = fmaxf(0.f, fmaxf(-lmL, -lmR));
        const float ssum = ap + am;
#pragma unroll
        for (int m = 0; m < 5; m++)
#pragma unroll
            for (int qq = 0; qq < 5; qq++) Fh[m][qq] = Fh[m + 1][qq];
        if (ssum > 0.f) {
            const float is = 1.f / ssum;
            const float wl = ap * is, wr = am * is, wd = ap * wr;
#pragma unroll
            for (int qq = 0; qq < 5; qq++)
                Fh[5][qq] = wl * FL[qq] + wr * FR[qq] - wd * (UR[qq] - UL[qq]);
        } else {
#pragma unroll
            for (int qq = 0; qq < 5; qq++) Fh[5][qq] = 0.5f * (FL[qq] + FR[qq]);
        }
        if (active) {
            // UCT face data: the two velocity components of both states, a+, a-
            // (each face once: the segment's own faces [k0, kend))
            if (f >= k0 && f < kend) {
                fd[fc] = L[1 + D];
                fd[n + fc] = L[1 + E1];
                fd[2 * n + fc] = R[1 + D];
                fd[3 * n + fc] = R[1 + E1];
                fd[4 * n + fc] = ap;
                fd[5 * n + fc] = am;
                if (owned(g, x, D == 1 ? wrapD(f) : o, D == 2 ? wrapD(f) : o))
                    amax = fmaxf(amax, fmaxf(ap, am));
            }
            // DER of cell f - 2 from faces f-5 .. f
            if (derc) {
#pragma unroll
                for (int qq = 0; qq < 5; qq++) {
                    const float s6[6] = {Fh[0][qq], Fh[1][qq], Fh[2][qq],
                                         Fh[3][qq], Fh[4][qq], Fh[5][qq]};
                    rhs[qq * n + cc] = der_sub(rh[qq], s6, w, g.ho);
                }
            }
        }
        __syncwarp();  // the queue of this face is read before the next face's entries
    }
    if (nfb && active) atomicAdd(&sc->rec_fallbacks, nfb);
    if (want_amax) {
        float m = warp_max_r(amax);
        if (lane == 0) red[warp] = m;
        __syncthreads();
        if (tid == 0) {
            float v = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
            const double vd = (double)v;
            if (vd > 0.0) atomicMax(&sc->amax_bits, (unsigned long long)__double_as_longlong(vd));
        }
    }
}

}  // namespace echo
