// Inversion fused with the x sweep, for the mixed path (Sec. 3, substep steps 1-3
// along x): INT + C2P of a row of cells, then MP5 reconstruction, physical fluxes,
// fast speeds and HLL at the row's faces, then the DER of those fluxes into the
// right-hand side, in one kernel.
//
// A block of 256 threads owns one row of nx cells along x (nx <= XS_NXMAX).  The
// row's float primitives and its face fluxes stay in shared memory between the
// phases (the primitives also go to global memory for the y and z sweeps), so the
// x sweep reads nothing back from HBM and no flux array is written.  The inversion
// is bound by the FP64 pipe and the sweep by FP32 issue: with three blocks
// resident per SM at different phases, the sweep of one row runs while the FP64
// pipe serves the inversion of another, which two separate kernels cannot do.
//
// The arithmetic per cell and per face is that of k_int_c2p<float> and
// k_flux<float, 0> + k_der<float, 0> (the same device functions); the row is
// periodic, as the grid is along x.
#pragma once

#include "echo_kernels.cuh"
#include "echo_sweep.cuh"

namespace echo {

constexpr int XS_BS = 256;
constexpr int XS_NXMAX = 1024;  // row cells in shared memory: 13 floats each

__host__ __device__ constexpr size_t xs_smem_bytes(int nx) { return (size_t)13 * nx * 4; }

// periodic index in the row for t in [-nx, 2 nx)
__device__ __forceinline__ int xs_wrap(int t, int nx)
{
    return t < 0 ? t + nx : (t >= nx ? t - nx : t);
}

__global__ void __launch_bounds__(XS_BS, 3)
k_c2p_xsweep(Grid g, const double *__restrict__ U, const double *__restrict__ Bf,
             double *__restrict__ W, float *__restrict__ prim, const float *__restrict__ Bf32,
             float *__restrict__ rhs, float *__restrict__ fd, C2PParams par, DevScalars *sc,
             int stage, int want_amax)
{
    extern __shared__ __align__(16) float xs[];  // P[8][nx], F[5][nx]
    __shared__ Mp5WarpQueue<14> wq[XS_BS / 32];
    __shared__ float red[XS_BS / 32];
    __shared__ int halted;
    // the flag may be raised by another block of this launch: read it once, so that
    // the whole block leaves or stays (the phases have block barriers)
    if (threadIdx.x == 0) halted = *(volatile int *)&sc->halt;
    __syncthreads();
    if (halted) return;
    const int nx = g.nx, tid = threadIdx.x, lane = tid & 31;
    const long n = g.n;
    const int j = (int)(blockIdx.x % (unsigned)g.ny), k = (int)(blockIdx.x / (unsigned)g.ny);
    const long row = ((long)k * g.ny + j) * nx;
    float *P = xs, *Fs = xs + 8 * nx;

    // ---- phase 1: INT + C2P of the row's cells (FP64) ----
    unsigned it = 0, it32 = 0, itm = 0, na = 0, nbad = 0;
    for (int i = tid; i < nx; i += XS_BS) {
        const long c = row + i;
        double u[5], B[3];
#pragma unroll
        for (int d = 0; d < 3; d++) B[d] = cell_field(g, Bf, c, i, j, k, d);
#pragma unroll
        for (int v = 0; v < 5; v++) u[v] = U[v * n + c];
        const C2PInv qi = c2p_invariants(u, B, g.gm1g, g.gm1g32);
        const double W0 = par.guess == 1 ? u[4] : W[c];
        double p[5], Wn;
        int iters, iters32;
        const bool bad = !c2p_newton<true>(qi, u, B, W0, par.tol, par.maxit, p, Wn, iters, par.pre32,
                                     iters32);
#pragma unroll
        for (int v = 0; v < 5; v++) {
            const float pv = to_f32(p[v]);
            P[v * nx + i] = pv;
            prim[v * n + c] = pv;
        }
#pragma unroll
        for (int v = 0; v < 3; v++) {
            const float bv = to_f32(B[v]);
            P[(5 + v) * nx + i] = bv;
            prim[(5 + v) * n + c] = bv;
        }
        W[c] = Wn;
        if (owned(g, i, j, k)) {
            it += (unsigned)iters;
            it32 += (unsigned)iters32;
            itm = itm > (unsigned)iters ? itm : (unsigned)iters;
            na++;
            nbad += bad ? 1u : 0u;
        }
    }
    {
        const unsigned s = __reduce_add_sync(0xffffffffu, it);
        const unsigned s32 = __reduce_add_sync(0xffffffffu, it32);
        const unsigned m = __reduce_max_sync(0xffffffffu, itm);
        const unsigned a = __reduce_add_sync(0xffffffffu, na);
        const unsigned b = __reduce_add_sync(0xffffffffu, nbad);
        if (lane == 0 && a) {
            atomicAdd(&sc->it_sum, (unsigned long long)s);
            if (s32) atomicAdd(&sc->it32_sum, (unsigned long long)s32);
            atomicAdd(&sc->c2p_calls, (unsigned long long)a);
            atomicMax(&sc->it_max, m);
            if (b) {
                atomicAdd(&sc->fails, b);
                if (atomicCAS(&sc->fail_stage, 0, stage) == 0) sc->fail_step = (long)sc->step;
                atomicOr(&sc->halt, 1);
            }
        }
    }
    __syncthreads();

    // ---- phase 2: REC + fluxes + HLL at the faces i + 1/2 (FP32) ----
    const float gam = g.gam32, gfac = g.gfac32;
    float amax = 0.f;
    unsigned nfb = 0;
    // The deferred MP5 limiting runs per warp (warp-synchronous queue, no block
    // barrier); every lane reconstructs, a lane past the row on the row's last face.
    Mp5WarpQueue<14> &q = wq[tid >> 5];
    for (int base = 0; base < nx; base += XS_BS) {
        const int i0 = base + tid;
        const bool active = i0 < nx;
        const int i = active ? i0 : nx - 1;
        int cs[6];
        float L[8], Rt[8];
        unsigned mask = 0;
        int cnt = 0;
#pragma unroll
        for (int m = 0; m < 6; m++) cs[m] = xs_wrap(i + m - 2, nx);
#pragma unroll
        for (int v = 0; v < 8; v++) {
            if (v == 5) continue;  // the normal field is the staggered face value
            const int kl = 2 * v - (v > 5 ? 2 : 0);
            float s[6];
#pragma unroll
            for (int m = 0; m < 6; m++) s[m] = P[v * nx + cs[m]];
            const float dc = s[3] - s[2];  // shared by both states of the face
            L[v] = q.defer(s[0], s[1], s[2], s[3], s[4], dc, kl, mask, lane, cnt);
            Rt[v] = q.defer(s[5], s[4], s[3], s[2], s[1], -dc, kl + 1, mask, lane, cnt);
        }
        __syncwarp();
        q.process(lane, cnt);
        __syncwarp();
#pragma unroll
        for (int v = 0; v < 8; v++) {
            if (v == 5) continue;
            const int kl = 2 * v - (v > 5 ? 2 : 0);
            if (mask & (1u << kl)) L[v] = q.get(kl, lane);
            if (mask & (1u << (kl + 1))) Rt[v] = q.get(kl + 1, lane);
        }
        __syncwarp();  // the queue of this batch is read before the next batch's entries
        if (active) {
            const long f = row + i;
            const float bn = Bf32[f];
            L[5] = bn;
            Rt[5] = bn;
            // positivity: reset a state to the first-order (cell) value
            int nf = 0;
            float v2L = L[1] * L[1] + L[2] * L[2] + L[3] * L[3];
            float v2R = Rt[1] * Rt[1] + Rt[2] * Rt[2] + Rt[3] * Rt[3];
            if (!(L[0] > 0.f) || !(L[4] > 0.f) || !(v2L < 1.f)) {
#pragma unroll
                for (int v = 0; v < 8; v++)
                    if (v != 5) L[v] = P[v * nx + cs[2]];
                v2L = L[1] * L[1] + L[2] * L[2] + L[3] * L[3];
                nf++;
            }
            if (!(Rt[0] > 0.f) || !(Rt[4] > 0.f) || !(v2R < 1.f)) {
#pragma unroll
                for (int v = 0; v < 8; v++)
                    if (v != 5) Rt[v] = P[v * nx + cs[3]];
                v2R = Rt[1] * Rt[1] + Rt[2] * Rt[2] + Rt[3] * Rt[3];
                nf++;
            }
            const bool own = owned(g, i, j, k);
            if (own) nfb += (unsigned)nf;
            float UL[8], FL[8], UR[8], FR[8], lmL, lpL, lmR, lpR;
            phys<float, 0>(L, v2L, gam, gfac, UL, FL, lmL, lpL);
            phys<float, 0>(Rt, v2R, gam, gfac, UR, FR, lmR, lpR);
            const float ap = rmax(0.f, rmax(lpL, lpR));
            const float am = rmax(0.f, rmax(-lmL, -lmR));
            const float s = ap + am;
            if (gtz(s)) {
                const float is = 1.f / s;
                const float wl = ap * is, wr = am * is, wd = ap * wr;
#pragma unroll
                for (int qq = 0; qq < 5; qq++)
                    Fs[qq * nx + i] = wl * FL[qq] + wr * FR[qq] - wd * (UR[qq] - UL[qq]);
            } else {
#pragma unroll
                for (int qq = 0; qq < 5; qq++) Fs[qq * nx + i] = 0.5f * (FL[qq] + FR[qq]);
            }
            // UCT face data: v_x and v_y of both states, a+, a-
            fd[f] = L[1];
            fd[n + f] = L[2];
            fd[2 * n + f] = Rt[1];
            fd[3 * n + f] = Rt[2];
            fd[4 * n + f] = ap;
            fd[5 * n + f] = am;
            if (own) amax = rmax(amax, rmax(ap, am));
        }
    }
    if (nfb) atomicAdd(&sc->rec_fallbacks, nfb);
    __syncthreads();

    // ---- phase 3: rhs = -DER_x(flux) of the row's cells ----
    const float *w = g.derw32[0];
    for (int i = tid; i < nx; i += XS_BS) {
        int fs[6];
#pragma unroll
        for (int m = 0; m < 6; m++) fs[m] = xs_wrap(i + m - 3, nx);  // faces i-5/2 .. i+5/2
        const long c = row + i;
#pragma unroll
        for (int qq = 0; qq < 5; qq++) {
            float s6[6];
#pragma unroll
            for (int m = 0; m < 6; m++) s6[m] = Fs[qq * nx + fs[m]];
            rhs[qq * n + c] = der_sub(0.f, s6, w, g.ho);
        }
    }
    if (want_amax) {
        const float m = warp_max_r(amax);
        if (lane == 0) red[tid >> 5] = m;
        __syncthreads();
        if (tid < 32) {
            float v = tid < XS_BS / 32 ? red[tid] : 0.f;
            v = warp_max_r(v);
            const double vd = (double)v;
            if (tid == 0 && vd > 0.0)
                atomicMax(&sc->amax_bits, (unsigned long long)__double_as_longlong(vd));
        }
    }
}

}  // namespace echo
