// Kernels of one Runge-Kutta substep, templated on the reconstruction precision R
// (double: FP64 path; float: mixed path).  Included by one translation unit per R.
//
// Work split (one thread per output value, x fastest so every stencil load of a
// warp is a contiguous 32-element row; the DER and UCT blocks cover 32 x 8 tiles,
// see tile_cell):
//   k_int_c2p   Sec. 3 step 1: INT of the staggered field + Newton inversion.
//   k_flux<D>   Sec. 3 step 2: MP5 of the 8 primitives at the face above each
//               cell along D, fluxes, fast speeds, HLL; UCT face data; max speed.
//   k_der<D>    Sec. 3 step 3: rhs -= DER_D(flux).
//   k_uct<C>    Sec. 3 step 4: four-state upwind edge field along C.
//   k_rk        Sec. 3 step 4 (curl with DER) + step 5 (SSP-RK3 stage).
#pragma once

#include "echo_internal.h"
#include "echo_mlp.cuh"

namespace echo {

constexpr int BS = 256;
// Resident blocks of 256 threads per SM asked of the compiler, per kernel and
// precision (measured on the 256^3 bench; 1 = no request).  The FP32 sweeps are
// issue- and latency-bound and gain from more warps despite a few spilled values
// (6 blocks at 40 registers: 5.3e8 -> 5.7e8 cell-updates/s against 4 blocks at 64);
// the FP32-path inversion and RK gain a little (3 %, 13 %).  The FP64 kernels are
// bound by the FP64 pipe; three blocks (at most 85 registers) keep the compiler
// from spending registers that would cost a block (flux sweep: 3 % faster).
constexpr int minb_flux(int rbytes) { return rbytes == 4 ? 6 : 3; }
constexpr int minb_uct(int rbytes) { return rbytes == 4 ? 6 : 3; }
constexpr int minb_c2p(int rbytes) { return rbytes == 4 ? 4 : 3; }
constexpr int minb_rk(int rbytes) { return rbytes == 4 ? 6 : 3; }

// Thread-to-cell maps of the sweeps.  T = 0: consecutive cells of the linear
// order.  T = 1 (2): a block is a 32 x 8 tile of the x-y (x-z) plane, one warp per
// row of 32 consecutive x; its 8 warps take 8 consecutive y (z) rows, so that a
// stencil along y (z) re-reads the rows its neighbour warps just loaded, from L1.
// A grid with fewer than 8 cells along the stacking direction (a 2-D grid, a thin
// block) would leave most warps of a tile idle: it takes the linear order.
template <int T> __host__ __device__ __forceinline__ bool tiled(const Grid &g)
{
    return T != 0 && (T == 1 ? g.ny : g.nz) >= 8;
}

template <int T>
__device__ __forceinline__ bool tile_cell(const Grid &g, int &i, int &j, int &k)
{
    if (!tiled<T>(g)) {
        const long c = blockIdx.x * (long)BS + threadIdx.x;
        if (c >= g.n) return false;
        coords(g, c, i, j, k);
        return true;
    }
    const int nT = T == 1 ? g.ny : g.nz;
    const unsigned nbx = (unsigned)(g.nx + 31) >> 5, nbt = (unsigned)(nT + 7) >> 3;
    unsigned b = blockIdx.x;
    const unsigned bx = b % nbx;
    b /= nbx;
    const unsigned bt = b % nbt, bo = b / nbt;
    i = (int)(32 * bx + (threadIdx.x & 31));
    const int t = (int)(8 * bt + (threadIdx.x >> 5));
    if (T == 1) {
        j = t;
        k = (int)bo;
    } else {
        k = t;
        j = (int)bo;
    }
    return i < g.nx && t < nT;
}

// blocks of the launch of a kernel with thread map T
template <int T> inline unsigned tile_blocks(const Grid &g)
{
    if (!tiled<T>(g)) return nblocks(g.n, BS);
    const unsigned nbx = (unsigned)(g.nx + 31) / 32;
    const unsigned nT = T == 1 ? g.ny : g.nz, no = T == 1 ? g.nz : g.ny;
    return nbx * ((nT + 7) / 8) * no;
}

// The map of each sweep (measured on the 256^3 bench): the DER of direction D
// stacks warps along D and the UCT of edge direction C along its b direction
// (C + 2) % 3 unless that is x (1-6 % faster each); the flux sweeps, whose many
// stencil loads per face already overlap within a block, keep the linear order
// (the tiles made them 2-4 % slower).
constexpr int flux_map(int) { return 0; }
constexpr int der_map(int D) { return D; }
constexpr int uct_map(int C) { return C == 2 ? 1 : 2; }

template <typename R>
__device__ __forceinline__ R ld(const R *p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// step 1: INT + C2P
// ---------------------------------------------------------------------------
// MLP: the learned starting guess is computed in the kernel from the cell's
// conserved state and field (the network's parameters mw in global memory, read
// through L1); a guess that is unusable falls back to the previous W and is counted.
// The network runs on whole warps, before the divergent Newton iteration: lanes
// past the grid evaluate it on a placeholder state.
// The network variant takes two blocks per SM (128 registers, no spills) on both
// paths: on a resume of the 128^3 turbulence its FP64 inversion took 1.25 ms with
// two blocks against 1.27 ms with three (spilling), the cold start 1.39 ms.
constexpr int minb_c2p_mlp(int) { return 2; }

template <typename R, bool MLP>
__global__ void __launch_bounds__(BS, MLP ? minb_c2p_mlp(sizeof(R)) : minb_c2p(sizeof(R)))
k_int_c2p(Grid g, const double *__restrict__ U, const double *__restrict__ Bf,
          double *__restrict__ W, const MlpDev *__restrict__ mw, R *__restrict__ prim,
          C2PParams par, DevScalars *sc, int stage, int update_w, int count)
{
    // the flag is set by other blocks of this launch: read it once per warp so that
    // the warp-wide reductions below always see all 32 lanes
    if (count && __reduce_or_sync(0xffffffffu, (unsigned)sc->halt)) return;
    const long n = g.n;
    long c = blockIdx.x * (long)BS + threadIdx.x;
    unsigned it = 0, it32 = 0;
    bool active = c < n, bad = false, fb = false, own = false;
    double u[5] = {1.0, 0.0, 0.0, 0.0, 2.0}, B[3] = {0.0, 0.0, 0.0};
    if (active) {
        int i, j, k;
        coords(g, c, i, j, k);
        own = owned(g, i, j, k);
#pragma unroll
        for (int d = 0; d < 3; d++) B[d] = cell_field(g, Bf, c, i, j, k, d);
#pragma unroll
        for (int v = 0; v < 5; v++) u[v] = U[v * n + c];
    }
    // the invariants serve the learned guess's features and the Newton iteration
    const C2PInv q = c2p_invariants(u, B, g.gm1g, g.gm1g32);
    double W0 = 0.0;
    if (MLP) {
        W0 = mlp_guess_warp(*mw, q, threadIdx.x & 31);
        // the conserved state is read again (from L1) rather than held in registers
        // across the network, whose fragments need them
        asm volatile("" ::: "memory");
        if (active)
#pragma unroll
            for (int v = 0; v < 5; v++) u[v] = U[v * n + c];
    }
    if (active) {
        // an unusable learned guess (outside W > 0, v^2 < 1) falls back to the previous
        // W inside the Newton routine's first evaluation, and is counted
        double Wfb = 0.0;
        if (MLP) Wfb = W[c];
        else if (par.guess == 1) W0 = u[4];
        else W0 = W[c];
        double p[5], Wn;
        int iters, iters32;
        // the FP32 pre-iterations and chord steps are compiled into the mixed path's
        // kernels only
        bad = !c2p_newton<sizeof(R) == 4>(q, u, B, W0, par.tol, par.maxit, p, Wn, iters,
                                          par.pre32, iters32, Wfb, MLP ? &fb : nullptr);
        it = (unsigned)iters;
        it32 = (unsigned)iters32;
#pragma unroll
        for (int v = 0; v < 5; v++) prim[v * n + c] = to_r<R>(p[v]);
#pragma unroll
        for (int v = 0; v < 3; v++) prim[(5 + v) * n + c] = to_r<R>(B[v]);
        if (update_w) W[c] = Wn;
        if (!own) {  // a neighbour's cell: updated, not counted
            it = it32 = 0;
            bad = fb = false;
        }
    }
    if (!count) return;
    unsigned s = __reduce_add_sync(0xffffffffu, it);
    unsigned s32 = __reduce_add_sync(0xffffffffu, it32);
    unsigned m = __reduce_max_sync(0xffffffffu, it);
    unsigned na = __popc(__ballot_sync(0xffffffffu, own));
    unsigned nb = __popc(__ballot_sync(0xffffffffu, bad));
    unsigned nf = __popc(__ballot_sync(0xffffffffu, fb));
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sc->it_sum, (unsigned long long)s);
        if (s32) atomicAdd(&sc->it32_sum, (unsigned long long)s32);
        atomicAdd(&sc->c2p_calls, (unsigned long long)na);
        atomicMax(&sc->it_max, m);
        if (nf) atomicAdd(&sc->fallbacks, nf);
        if (nb) {
            atomicAdd(&sc->fails, nb);
            // the step in progress is the count of completed ones
            if (atomicCAS(&sc->fail_stage, 0, stage) == 0) sc->fail_step = (long)sc->step;
            atomicOr(&sc->halt, 1);
        }
    }
}

// Learned Newton starting guesses W0 = U y of every cell into guess[n] (the values
// the inversion kernel computes in place; used by echo_mlp_guess).  Persistent
// blocks: the weights go to shared memory once per block, which then walks the grid
// in steps of the whole launch.  BT: precision of the face field read for the
// features (the float mirror on the mixed path, as in the step).
constexpr int MLP_BS = 128;

template <typename BT>
__global__ void __launch_bounds__(MLP_BS)
k_mlp_guess(Grid g, const double *__restrict__ U, const BT *__restrict__ Bf,
            const MlpDev *__restrict__ w, double *__restrict__ guess)
{
    __shared__ __align__(16) unsigned char smem[MLP_INFER_BYTES];
    const MlpDev &sw = load_mlp_shared(smem, w);
    const int lane = threadIdx.x & 31;
    const long n = g.n;
    for (long base = blockIdx.x * (long)MLP_BS; base < n; base += (long)gridDim.x * MLP_BS) {
        const long c = base + threadIdx.x;
        double u[5] = {1.0, 0.0, 0.0, 0.0, 2.0}, B[3] = {0.0, 0.0, 0.0};
        if (c < n) {
            int i, j, k;
            coords(g, c, i, j, k);
            for (int d = 0; d < 3; d++) B[d] = cell_field(g, Bf, c, i, j, k, d);
            for (int v = 0; v < 5; v++) u[v] = U[v * n + c];
        }
        const double w0 = mlp_guess_warp(sw, c2p_invariants(u, B, g.gm1g, g.gm1g32), lane);
        if (c < n) guess[c] = w0;
    }
}

// ---------------------------------------------------------------------------
// steps 2: reconstruction + HLL at the faces along D
// ---------------------------------------------------------------------------
// queue capacity of the deferred MP5 limiting: two entries per thread on average
constexpr int QMAX = 2 * BS;


template <typename R, int D>
__global__ void __launch_bounds__(BS, minb_flux(sizeof(R)))
k_flux(Grid g, const R *__restrict__ prim, const R *__restrict__ Bf, R *__restrict__ flux,
       R *__restrict__ fd, DevScalars *sc, int want_amax)
{
    if (sc->halt) return;
    __shared__ Mp5Queue<R, 16, QMAX, BS> q;
    q.reset();
    __syncthreads();
    const long n = g.n;
    const int uct = g.uct;
    int i, j, k;
    const bool active = tile_cell<flux_map(D)>(g, i, j, k);
    const long f = active ? ((long)k * g.ny + j) * g.nx + i : 0;
    R amax = R(0);
    int cs[6];
    R L[8], Rt[8];
    unsigned mask = 0;
    bool own = false;  // face i+1/2 belongs to cell i
    if (active) {
        own = owned(g, i, j, k);
        const int iD = D == 0 ? i : (D == 1 ? j : k);
#pragma unroll
        for (int m = 0; m < 6; m++) cs[m] = sidx<D>(g, (int)f, iD, m - 2);
#pragma unroll
        for (int v = 0; v < 8; v++) {
            // with UCT the normal field is the staggered face value, not reconstructed
            if (v == 5 + D && uct) continue;
            R s[6];
            const R *pv = prim + v * n;
            if (g.rec) {  // linear: cells i-1 .. i+2
#pragma unroll
                for (int m = 1; m < 5; m++) s[m] = ld(pv + cs[m]);
                L[v] = mc_val(s[1], s[2], s[3]);
                Rt[v] = mc_val(s[4], s[3], s[2]);
            } else {
#pragma unroll
                for (int m = 0; m < 6; m++) s[m] = ld(pv + cs[m]);
                const R dc = s[3] - s[2];  // shared by both states of the face
                L[v] = q.defer(s[0], s[1], s[2], s[3], s[4], dc, 2 * v, mask);
                Rt[v] = q.defer(s[5], s[4], s[3], s[2], s[1], -dc, 2 * v + 1, mask);
            }
        }
    }
    __syncthreads();
    q.process();
    __syncthreads();
    if (active) {
#pragma unroll
        for (int v = 0; v < 8; v++) {
            if (mask & (1u << (2 * v))) L[v] = q.get(2 * v);
            if (mask & (1u << (2 * v + 1))) Rt[v] = q.get(2 * v + 1);
        }
        if (uct) {
            const R bn = Bf[D * n + f];
            L[5 + D] = bn;
            Rt[5 + D] = bn;
        }
        // positivity: reset a state to the first-order (cell) value
        int nfb = 0;
        R v2L = L[1] * L[1] + L[2] * L[2] + L[3] * L[3];
        R v2R = Rt[1] * Rt[1] + Rt[2] * Rt[2] + Rt[3] * Rt[3];
        if (!gtz(L[0]) || !gtz(L[4]) || !lt(v2L, R(1))) {
#pragma unroll
            for (int v = 0; v < 8; v++)
                if (v != 5 + D || !uct) L[v] = prim[v * n + cs[2]];
            v2L = L[1] * L[1] + L[2] * L[2] + L[3] * L[3];
            nfb++;
        }
        if (!gtz(Rt[0]) || !gtz(Rt[4]) || !lt(v2R, R(1))) {
#pragma unroll
            for (int v = 0; v < 8; v++)
                if (v != 5 + D || !uct) Rt[v] = prim[v * n + cs[3]];
            v2R = Rt[1] * Rt[1] + Rt[2] * Rt[2] + Rt[3] * Rt[3];
            nfb++;
        }
        if (nfb && own) atomicAdd(&sc->rec_fallbacks, (unsigned)nfb);
        const R gam = gconst<R>(g.gam, g.gam32);
        const R gfac = gconst<R>(g.gfac, g.gfac32);
        R UL[8], FL[8], UR[8], FR[8], lmL, lpL, lmR, lpR;
        phys<R, D>(L, v2L, gam, gfac, UL, FL, lmL, lpL);
        phys<R, D>(Rt, v2R, gam, gfac, UR, FR, lmR, lpR);
        R ap = rmax(R(0), rmax(lpL, lpR));
        R am = rmax(R(0), rmax(-lmL, -lmR));
        R s = ap + am;
        const int ncomp = uct ? 5 : 8;  // with UCT the field takes the edge fields instead
        if (gtz(s)) {
            // HLL weights divided once: a+/(a+ + a-), a-/(a+ + a-), a+ a-/(a+ + a-)
            const R is = rcp_r(s);
            const R wl = ap * is, wr = am * is, wd = ap * wr;
#pragma unroll
            for (int qq = 0; qq < 8; qq++)
                if (qq < ncomp)
                    flux[qq * n + f] = wl * FL[qq] + wr * FR[qq] - wd * (UR[qq] - UL[qq]);
        } else {
#pragma unroll
            for (int qq = 0; qq < 8; qq++)
                if (qq < ncomp) flux[qq * n + f] = R(0.5) * (FL[qq] + FR[qq]);
        }
        if (uct) {
            constexpr int E1 = (D + 1) % 3;
            fd[f] = L[1 + D];
            fd[n + f] = L[1 + E1];
            fd[2 * n + f] = Rt[1 + D];
            fd[3 * n + f] = Rt[1 + E1];
            fd[4 * n + f] = ap;
            fd[5 * n + f] = am;
        }
        if (own) amax = rmax(ap, am);
    }
    if (want_amax) {
        // block maximum in R (non-negative values), one conversion per block
        __shared__ R red[BS / 32];
        R m = warp_max_r(amax);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x < 32) {
            R v = threadIdx.x < BS / 32 ? red[threadIdx.x] : R(0);
            v = warp_max_r(v);
            const double vd = (double)v;
            if (threadIdx.x == 0 && vd > 0.0)
                atomicMax(&sc->amax_bits, (unsigned long long)__double_as_longlong(vd));
        }
    }
}

// ---------------------------------------------------------------------------
// step 3: rhs -= DER_D(flux)
// ---------------------------------------------------------------------------
template <typename R, int D>
__global__ void __launch_bounds__(BS)
k_der(Grid g, const R *__restrict__ flux, R *__restrict__ rhs, int first, DevScalars *sc)
{
    if (sc->halt) return;
    const long n = g.n;
    int i, j, k;
    if (!tile_cell<der_map(D)>(g, i, j, k)) return;
    const long c = ((long)k * g.ny + j) * g.nx + i;
    const int iD = D == 0 ? i : (D == 1 ? j : k);
    int fs[6];
#pragma unroll
    for (int m = 0; m < 6; m++) fs[m] = sidx<D>(g, (int)c, iD, m - 3);
    const R *w = derw<R>(g, D);
    const int ncomp = g.uct ? 5 : 8;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        if (q >= ncomp) break;
        R s[6];
#pragma unroll
        for (int m = 0; m < 6; m++) s[m] = ld(flux + q * n + (long)fs[m]);
        rhs[q * n + c] = der_sub(first ? R(0) : rhs[q * n + c], s, w, g.ho);
    }
}

// ---------------------------------------------------------------------------
// step 4a: UCT edge field along C
// ---------------------------------------------------------------------------
template <typename R, int C>
__global__ void __launch_bounds__(BS, minb_uct(sizeof(R)))
k_uct(Grid g, const R *__restrict__ Bf, const R *__restrict__ fda, const R *__restrict__ fdb,
      R *__restrict__ E, DevScalars *sc)
{
    if (sc->halt) return;
    constexpr int A = (C + 1) % 3, B = (C + 2) % 3;
    __shared__ Mp5Queue<R, 12, QMAX, BS> q;
    q.reset();
    __syncthreads();
    const long n = g.n;
    int i, j, k;
    const bool active = tile_cell<uct_map(C)>(g, i, j, k);
    const long e = active ? ((long)k * g.ny + j) * g.nx + i : 0;
    // slots: va[s][t] = 4 s + t, vb[s][t] = 4 s + 2 + t, Ba[t] = 8 + t, Bb[s] = 10 + s
    R r[12];
    unsigned mask = 0;
    int sb[6], sa[6];
    const int lin = g.rec;
    // left/right states of one stencil into slots k, k+1 of r
    auto recon = [&](const R *s, int k) {
        if (lin) {
            r[k] = mc_val(s[1], s[2], s[3]);
            r[k + 1] = mc_val(s[4], s[3], s[2]);
        } else {
            const R dc = s[3] - s[2];  // shared by both states
            r[k] = q.defer(s[0], s[1], s[2], s[3], s[4], dc, k, mask);
            r[k + 1] = q.defer(s[5], s[4], s[3], s[2], s[1], -dc, k + 1, mask);
        }
    };
    if (active) {
        const int iA = A == 0 ? i : (A == 1 ? j : k), iB = B == 0 ? i : (B == 1 ? j : k);
#pragma unroll
        for (int m = 0; m < 6; m++) {
            sb[m] = sidx<B>(g, (int)e, iB, m - 2);
            sa[m] = sidx<A>(g, (int)e, iA, m - 2);
        }
        R s[6];
#pragma unroll
        for (int qs = 0; qs < 2; qs++) {
#pragma unroll
            for (int m = 0; m < 6; m++) s[m] = ld(fda + (2 * qs) * n + sb[m]);
            recon(s, 4 * qs + 0);
#pragma unroll
            for (int m = 0; m < 6; m++) s[m] = ld(fda + (2 * qs + 1) * n + sb[m]);
            recon(s, 4 * qs + 2);
        }
#pragma unroll
        for (int m = 0; m < 6; m++) s[m] = ld(Bf + A * n + sb[m]);
        recon(s, 8);
#pragma unroll
        for (int m = 0; m < 6; m++) s[m] = ld(Bf + B * n + sa[m]);
        recon(s, 10);
    }
    __syncthreads();
    q.process();
    __syncthreads();
    if (!active) return;
#pragma unroll
    for (int k2 = 0; k2 < 12; k2++)
        if (mask & (1u << k2)) r[k2] = q.get(k2);
    R va[2][2] = {{r[0], r[1]}, {r[4], r[5]}};
    R vb[2][2] = {{r[2], r[3]}, {r[6], r[7]}};
    R Ba[2] = {r[8], r[9]}, Bb[2] = {r[10], r[11]};
    R apa = rmax(ld(fda + 4 * n + e), ld(fda + 4 * n + sb[3]));
    R ama = rmax(ld(fda + 5 * n + e), ld(fda + 5 * n + sb[3]));
    R apb = rmax(ld(fdb + 4 * n + e), ld(fdb + 4 * n + sa[3]));
    R amb = rmax(ld(fdb + 5 * n + e), ld(fdb + 5 * n + sa[3]));
    E[C * n + e] = uct_point(va, vb, Ba, Bb, apa, ama, apb, amb);
}

// minus the curl of the edge field on the a-faces of cell (i,j,k), i.e. dB_a/dt:
// D_c E_b - D_b E_c
template <typename R>
__device__ __forceinline__ R neg_curl_a(const Grid &g, const R *__restrict__ E, int a, int i,
                                        int j, int k)
{
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    const long n = g.n;
    R s[6], t[6];
#pragma unroll
    for (int m = 0; m < 6; m++) {
        s[m] = ld(E + c * n + shifted_rt(g, i, j, k, b, m - 3));
        t[m] = ld(E + b * n + shifted_rt(g, i, j, k, c, m - 3));
    }
    return der_add(der_sub(R(0), s, derw<R>(g, b), g.ho), t, derw<R>(g, c), g.ho);
}

// ---------------------------------------------------------------------------
// step 4b + 5: curl of E and the SSP-RK3 stage on 5 cell + 3 face variables
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(BS, minb_rk(sizeof(R)))
k_rk(Grid g, int stage, int last, double a0, const R *__restrict__ E, const R *__restrict__ rhs,
     double *__restrict__ U, double *__restrict__ U0, double *__restrict__ Bf,
     double *__restrict__ Bf0, float *__restrict__ Bf32, DevScalars *sc)
{
    if (sc->halt) return;
    const long n = g.n;
    long c = blockIdx.x * (long)BS + threadIdx.x;
    const double dt = sc->dt;
    // Mixed path: L is an FP32 result, so its stage increment (1 - a0) dt L is formed
    // in FP32 (one rounding of the size of L's own) and widened; the combination with
    // U and the stage's base state stays FP64 -- two FP64 operations per variable
    // instead of three.
    const double c1 = 1.0 - a0;
    const float cinc = sizeof(R) == 4 ? to_f32(stage == 1 ? dt : c1 * dt) : 0.f;
    if (c < n) {
        int i, j, k;
        coords(g, c, i, j, k);
#pragma unroll
        for (int v = 0; v < 8; v++) {
            R rr;
            double u, *pu, *pu0;
            if (v < 5) {
                rr = rhs[v * n + c];
                pu = U + v * n + c;
                pu0 = U0 + v * n + c;
            } else {
                rr = g.uct ? neg_curl_a(g, E, v - 5, i, j, k) : rhs[v * n + c];
                pu = Bf + (v - 5) * n + c;
                pu0 = Bf0 + (v - 5) * n + c;
            }
            u = *pu;
            // stage 1: U1 = Un + dt L; later stages: a0 Un + (1 - a0) (U + dt L)
            // (SSP-RK3: a0 = 3/4, 1/3; SSP-RK2: a0 = 1/2)
            double un;
            if constexpr (sizeof(R) == 4) {
                const double inc = to_f64(cinc * rr);
                if (stage == 1) {
                    *pu0 = u;
                    un = u + inc;
                } else {
                    un = (*pu0) * a0 + (c1 * u + inc);
                }
            } else {
                const double r = to_f64(rr);
                if (stage == 1) {
                    *pu0 = u;
                    un = u + dt * r;
                } else {
                    un = (*pu0) * a0 + c1 * (u + dt * r);
                }
            }
            *pu = un;
            if (v >= 5 && Bf32) Bf32[(v - 5) * n + c] = to_f32(un);
        }
    }
    if (last && g.primary && blockIdx.x == 0 && threadIdx.x == 0) sc->step += 1;
}

// out (double) = sign * curl(E) on faces, accumulate or overwrite
template <typename R>
__global__ void __launch_bounds__(BS)
k_curl(Grid g, const R *__restrict__ E, double *__restrict__ out, double sign, int accumulate)
{
    const long n = g.n;
    long c = blockIdx.x * (long)BS + threadIdx.x;
    if (c >= n) return;
    int i, j, k;
    coords(g, c, i, j, k);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        double v = -sign * to_f64(neg_curl_a(g, E, a, i, j, k));
        out[a * n + c] = accumulate ? out[a * n + c] + v : v;
    }
}

template <typename R>
__global__ void __launch_bounds__(BS) k_to_double(long m, const R *__restrict__ in, double *__restrict__ out)
{
    long q = blockIdx.x * (long)BS + threadIdx.x;
    if (q < m) out[q] = to_f64(in[q]);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// the face field in R: the double state itself, or its float mirror
template <typename R> inline const R *face_field(echo_ctx *c);
template <> inline const double *face_field<double>(echo_ctx *c) { return c->Bf; }
template <> inline const float *face_field<float>(echo_ctx *c) { return c->Bf32; }

template <typename R>
void Path<R>::int_c2p(echo_ctx *c, int stage, int update_w, bool learned)
{
    // the mixed path refines the guess with FP32 Newton iterations first
    C2PParams par{c->cfg.c2p_tol, c->cfg.c2p_maxit, c->cfg.c2p_guess, c->mixed ? 1 : 0};
    const bool mlp = learned && c->mlp_w;
    if (par.guess == ECHO_GUESS_MLP) par.guess = ECHO_GUESS_PREV;
    if (mlp)
        launch(c, K_C2P, k_int_c2p<R, true>, nblocks(c->g.n, BS), BS, 0, c->g,
               (const double *)c->U, (const double *)c->Bf, c->W, (const MlpDev *)c->mlp_w,
               (R *)c->prim, par, c->sc, stage, update_w, 1);
    else
        launch(c, K_C2P, k_int_c2p<R, false>, nblocks(c->g.n, BS), BS, 0, c->g,
               (const double *)c->U, (const double *)c->Bf, c->W, (const MlpDev *)nullptr,
               (R *)c->prim, par, c->sc, stage, update_w, 1);
}

template <typename R>
void Path<R>::mlp_guess(echo_ctx *c)
{
    // persistent grid: as many blocks as can be resident at once (sized when the
    // weights were loaded)
    unsigned nb = nblocks(c->g.n, MLP_BS);
    if (c->mlp_blocks && nb > c->mlp_blocks) nb = c->mlp_blocks;
    launch(c, K_MLP, k_mlp_guess<R>, nb, MLP_BS, 0, c->g, (const double *)c->U, face_field<R>(c),
           (const MlpDev *)c->mlp_w, c->guess);
}

template <typename R>
unsigned Path<R>::mlp_grid(echo_ctx *c)
{
    int nsm = 152, per_sm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->cfg.device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_guess<R>, MLP_BS, 0);
    return (unsigned)(nsm * (per_sm > 0 ? per_sm : 1));
}

template <typename R>
void Path<R>::c2p_sweeps(echo_ctx *c, int stage, bool learned, int want_amax)
{
    if (sizeof(R) == 4 && c->xsweep && !(learned && c->mlp_w)) {
        launch_c2p_xsweep(c, stage, want_amax);
        sweeps(c, want_amax, 0);
    } else {
        int_c2p(c, stage, 1, learned);
        sweeps(c, want_amax, 1);
    }
}

template <typename R>
void Path<R>::sweeps(echo_ctx *c, int want_amax, int with_x)
{
    const Grid &g = c->g;
    const unsigned nb0 = tile_blocks<flux_map(0)>(g), nb1 = tile_blocks<flux_map(1)>(g),
                   nb2 = tile_blocks<flux_map(2)>(g);
    const unsigned nd0 = tile_blocks<der_map(0)>(g), nd1 = tile_blocks<der_map(1)>(g),
                   nd2 = tile_blocks<der_map(2)>(g);
    const R *prim = (const R *)c->prim;
    const R *bf = face_field<R>(c);
    R *flux = (R *)c->flux, *rhs = (R *)c->rhs;
    if (with_x) {
        launch(c, K_FLUX_X, k_flux<R, 0>, nb0, BS, 0, g, prim, bf, flux,
               (R *)c->fdat[0], c->sc, want_amax);
        launch(c, K_DER_X, k_der<R, 0>, nd0, BS, 0, g, (const R *)flux, rhs, 1, c->sc);
    }
    // mixed path: y and z as fused sweeps where chosen (TMA-staged planes, the face
    // fluxes kept on chip), else the flux kernel and its DER
    if (sizeof(R) == 4 && c->sweep_T[1]) {
        launch_fused_sweep(c, 1, want_amax);
    } else {
        launch(c, K_FLUX_Y, k_flux<R, 1>, nb1, BS, 0, g, prim, bf, flux,
               (R *)c->fdat[1], c->sc, want_amax);
        launch(c, K_DER_Y, k_der<R, 1>, nd1, BS, 0, g, (const R *)flux, rhs, 0, c->sc);
    }
    if (sizeof(R) == 4 && c->sweep_T[2]) {
        launch_fused_sweep(c, 2, want_amax);
    } else {
        launch(c, K_FLUX_Z, k_flux<R, 2>, nb2, BS, 0, g, prim, bf, flux,
               (R *)c->fdat[2], c->sc, want_amax);
        launch(c, K_DER_Z, k_der<R, 2>, nd2, BS, 0, g, (const R *)flux, rhs, 0, c->sc);
    }
}

template <typename R>
void Path<R>::uct(echo_ctx *c)
{
    if (!c->g.uct) return;
    const Grid &g = c->g;
    const R *f0 = (const R *)c->fdat[0], *f1 = (const R *)c->fdat[1], *f2 = (const R *)c->fdat[2];
    const R *bf = face_field<R>(c);
    // E_z from x-faces (a) and y-faces (b); E_x from y and z; E_y from z and x
    launch(c, K_UCT_Z, k_uct<R, 2>, tile_blocks<uct_map(2)>(g), BS, 0, g, bf, f0, f1, (R *)c->E,
           c->sc);
    launch(c, K_UCT_X, k_uct<R, 0>, tile_blocks<uct_map(0)>(g), BS, 0, g, bf, f1, f2, (R *)c->E,
           c->sc);
    launch(c, K_UCT_Y, k_uct<R, 1>, tile_blocks<uct_map(1)>(g), BS, 0, g, bf, f2, f0, (R *)c->E,
           c->sc);
}

template <typename R>
void Path<R>::rk(echo_ctx *c, int stage)
{
    const int order = c->cfg.rk_order;
    const double a0 = order == 2 ? 0.5 : (stage == 2 ? 0.75 : 1.0 / 3.0);
    launch(c, K_RK, k_rk<R>, nblocks(c->g.n, BS), BS, 0, c->g, stage, stage == order ? 1 : 0, a0,
           (const R *)c->E,
           (const R *)c->rhs, c->U, c->U0, c->Bf, c->Bf0, c->Bf32, c->sc);
}

template <typename R>
void Path<R>::curl_out(echo_ctx *c, double *out)
{
    launch(c, K_CURL, k_curl<R>, nblocks(c->g.n, BS), BS, 0, c->g, (const R *)c->E, out, -1.0, 0);
}

template <typename R>
void Path<R>::rhs_out(echo_ctx *c, double *out)
{
    long m = (c->g.uct ? 5 : 8) * c->g.n;
    launch(c, K_MISC, k_to_double<R>, nblocks(m, BS), BS, 0, m, (const R *)c->rhs, out);
}

}  // namespace echo
