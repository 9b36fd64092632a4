/*
 * Plain, slow FP64 CPU oracle for the ECHO special-relativistic MHD right-hand-side
 * update (arXiv 2401.03008).  TEST INFRASTRUCTURE ONLY: it is called by the tests,
 * by the smoke check and by the CPU-baseline leg of the benchmark, never by the
 * product path.  It shares no code, header or constant with the CUDA library.
 *
 * Everything is double precision and written in the order the paper lists the
 * steps of one Runge-Kutta substep (Sec. 3, steps 1-5):
 *   1. INT of the staggered field to cell centres, then the Newton C2P inversion;
 *   2. REC (MP5) of primitives at every interface, physical fluxes, HLL flux,
 *      fast speeds and the face data needed by UCT;
 *   3. DER of the numerical fluxes (flat space, Sec. 2: every source term of
 *      Eq. 4 holds a metric derivative, so none remains);
 *   4. UCT edge electric fields and their curl (DER again);
 *   5. the Runge-Kutta stage update and, once per step, the timestep.
 * Where the paper only names a method, the textbook form used here is stated at
 * the function that implements it.
 *
 * Layout: every grid array is [var][nz][ny][nx] with x fastest, periodic in all
 * directions, no ghost cells (indices wrap).  Cell (i,j,k) sits at
 * ((i+1/2)hx, (j+1/2)hy, (k+1/2)hz).  A face array of direction d stores at index
 * (i,j,k) the value on the face half a cell above the cell centre along d; an
 * edge array of direction c stores the value at the edge half a cell above the
 * cell centre along both directions other than c.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction, so
 * every product is rounded as written).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Configuration and statistics                                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
    double gam;          /* adiabatic index of the ideal-gas law (Sec. 2, Eq. 6) */
    double cfl;
    int uct;             /* 1: staggered B evolved by UCT; 0: cell-centred B */
    int ho;              /* 1: high-order INT and DER; 0: two-point forms */
    double tol;          /* Newton stop: |dW| <= tol*W */
    int maxit;           /* Newton iteration cap */
    int guess;           /* 0: previous W (warm), 1: W0 = U (cold), 2: caller array */
    int nthreads;        /* OpenMP threads (0: library default) */
    int rec;             /* 0: MP5; 1: linear with the MC limiter */
    int rk;              /* Runge-Kutta order: 3 (SSP-RK3) or 2 (SSP-RK2) */
} orc_cfg;

typedef struct {
    long cells;          /* C2P calls */
    long iters;          /* Newton iterations summed over calls */
    int itmax;           /* largest iteration count of one call */
    long failures;       /* calls that did not converge or gave an unphysical state */
    long fallbacks;      /* caller guesses rejected as unphysical */
    long rec_fallbacks;  /* interface states reset to first order */
} orc_stats;

#define MP5_ALPHA 4.0
#define MP5_EPS 1e-10

static double sq(double x) { return x * x; }

static int wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* linear index of cell (i,j,k) moved by s cells along direction d */
static long at(const orc_cfg *g, int i, int j, int k, int d, int s)
{
    if (d == 0) i += s;
    else if (d == 1) j += s;
    else k += s;
    i = wrap(i, g->nx);
    j = wrap(j, g->ny);
    k = wrap(k, g->nz);
    return ((long)k * g->ny + j) * g->nx + i;
}

static long ncell(const orc_cfg *g) { return (long)g->nx * g->ny * g->nz; }

static double hdir(const orc_cfg *g, int d)
{
    return d == 0 ? g->lx / g->nx : (d == 1 ? g->ly / g->ny : g->lz / g->nz);
}

static void set_threads(const orc_cfg *g)
{
#ifdef _OPENMP
    if (g->nthreads > 0) omp_set_num_threads(g->nthreads);
#else
    (void)g;
#endif
}

/* ------------------------------------------------------------------------- */
/* Point-wise physics (Sec. 2, flat space, ideal MHD)                        */
/* ------------------------------------------------------------------------- */

/* Ideal MHD closure E = -v x B (Sec. 2, text before Eq. 8). */
static void efield(const double *v, const double *B, double *E)
{
    E[0] = -(v[1] * B[2] - v[2] * B[1]);
    E[1] = -(v[2] * B[0] - v[0] * B[2]);
    E[2] = -(v[0] * B[1] - v[1] * B[0]);
}

/* Conserved variables from primitives (Sec. 2 definitions after Eq. 5 and the
 * ideal-gas enthalpy Eq. 6): D = rho*G, S = rho*h*G^2 v + E x B,
 * U = rho*h*G^2 - p + (E^2+B^2)/2.  prim = (rho, vx, vy, vz, p). */
void orc_prim2cons(const double *prim, const double *B, double gam, double *u)
{
    double v[3] = {prim[1], prim[2], prim[3]};
    double rho = prim[0], p = prim[4];
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double lor2 = 1.0 / (1.0 - v2);
    double lor = sqrt(lor2);
    double rhoh = rho + gam / (gam - 1.0) * p;
    double w = rhoh * lor2;
    double E[3];
    efield(v, B, E);
    double e2 = E[0] * E[0] + E[1] * E[1] + E[2] * E[2];
    double b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    u[0] = rho * lor;
    u[1] = w * v[0] + (E[1] * B[2] - E[2] * B[1]);
    u[2] = w * v[1] + (E[2] * B[0] - E[0] * B[2]);
    u[3] = w * v[2] + (E[0] * B[1] - E[1] * B[0]);
    u[4] = w - p + 0.5 * (e2 + b2);
}

/* Physical flux along d of the 8 conserved quantities (D, Sx, Sy, Sz, U, Bx, By, Bz)
 * from the divergence form Eq. 8: F(D) = D v_d,
 * F(S_i) = rho h G^2 v_i v_d - E_i E_d - B_i B_d + p_tot delta_id, F(U) = S_d,
 * F(B_i) = v_d B_i - v_i B_d (the curl term written as a flux). */
void orc_flux(const double *prim, const double *B, double gam, int d, double *f)
{
    double v[3] = {prim[1], prim[2], prim[3]};
    double rho = prim[0], p = prim[4];
    double u[5];
    orc_prim2cons(prim, B, gam, u);
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double lor2 = 1.0 / (1.0 - v2);
    double w = (rho + gam / (gam - 1.0) * p) * lor2;
    double E[3];
    efield(v, B, E);
    double ptot = p + 0.5 * (E[0] * E[0] + E[1] * E[1] + E[2] * E[2] +
                             B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    f[0] = u[0] * v[d];
    for (int i = 0; i < 3; i++)
        f[1 + i] = w * v[i] * v[d] - E[i] * E[d] - B[i] * B[d] + (i == d ? ptot : 0.0);
    f[4] = u[1 + d];
    for (int i = 0; i < 3; i++)
        f[5 + i] = v[d] * B[i] - v[i] * B[d];
}

/* Fastest characteristic speeds along d.  The paper only says that fast speeds are
 * computed and stored (Sec. 3, step 2); this is the published approximate
 * fast-magnetosonic form for ideal RMHD: cs^2 = gam p/(rho h),
 * b^2 = B^2/G^2 + (v.B)^2, ca^2 = b^2/(rho h + b^2), w^2 = cs^2 + ca^2 - cs^2 ca^2,
 * lam(+-) = [v_d (1-w^2) +- sqrt(w^2 (1-v^2) ((1 - v^2 w^2) - v_d^2 (1-w^2)))]
 *           / (1 - v^2 w^2). */
void orc_speeds(const double *prim, const double *B, double gam, int d,
                double *lm, double *lp)
{
    double v[3] = {prim[1], prim[2], prim[3]};
    double rho = prim[0], p = prim[4];
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double rhoh = rho + gam / (gam - 1.0) * p;
    double cs2 = gam * p / rhoh;
    double vb = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
    double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double b2 = B2 * (1.0 - v2) + vb * vb;
    double ca2 = b2 / (rhoh + b2);
    double w2 = cs2 + ca2 - cs2 * ca2;
    double vd = v[d];
    double disc = w2 * (1.0 - v2) * ((1.0 - v2 * w2) - vd * vd * (1.0 - w2));
    if (disc < 0.0) disc = 0.0;
    double den = 1.0 - v2 * w2;
    double sr = sqrt(disc);
    *lp = (vd * (1.0 - w2) + sr) / den;
    *lm = (vd * (1.0 - w2) - sr) / den;
}

/* HLL numerical flux (Sec. 3 step 2, "second order approximation of the
 * point-value numerical flux" from left/right states): a+ = max(0, lp_L, lp_R),
 * a- = max(0, -lm_L, -lm_R),
 * F = (a+ F_L + a- F_R - a+ a- (U_R - U_L)) / (a+ + a-);
 * if a+ + a- = 0 the mean of F_L and F_R.  All 8 components; the caller keeps the
 * ones it needs. */
void orc_hll(const double *pL, const double *BL, const double *pR, const double *BR,
             double gam, int d, double *fhat, double *ap_out, double *am_out)
{
    double fL[8], fR[8], uL[5], uR[5], lmL, lpL, lmR, lpR;
    orc_flux(pL, BL, gam, d, fL);
    orc_flux(pR, BR, gam, d, fR);
    orc_prim2cons(pL, BL, gam, uL);
    orc_prim2cons(pR, BR, gam, uR);
    orc_speeds(pL, BL, gam, d, &lmL, &lpL);
    orc_speeds(pR, BR, gam, d, &lmR, &lpR);
    double ap = fmax(0.0, fmax(lpL, lpR));
    double am = fmax(0.0, fmax(-lmL, -lmR));
    double qL[8], qR[8];
    for (int c = 0; c < 5; c++) { qL[c] = uL[c]; qR[c] = uR[c]; }
    for (int c = 0; c < 3; c++) { qL[5 + c] = BL[c]; qR[5 + c] = BR[c]; }
    double s = ap + am;
    for (int c = 0; c < 8; c++) {
        if (s > 0.0)
            fhat[c] = (ap * fL[c] + am * fR[c] - ap * am * (qR[c] - qL[c])) / s;
        else
            fhat[c] = 0.5 * (fL[c] + fR[c]);
    }
    *ap_out = ap;
    *am_out = am;
}

/* ------------------------------------------------------------------------- */
/* High-order 1-D operators on stencils (the paper's REC, INT, DER; Sec. 3)  */
/* ------------------------------------------------------------------------- */

static double minmod2(double a, double b)
{
    if (a > 0.0 && b > 0.0) return fmin(a, b);
    if (a < 0.0 && b < 0.0) return fmax(a, b);
    return 0.0;
}

static double minmod4(double a, double b, double c, double d)
{
    if (a > 0.0 && b > 0.0 && c > 0.0 && d > 0.0) return fmin(fmin(a, b), fmin(c, d));
    if (a < 0.0 && b < 0.0 && c < 0.0 && d < 0.0) return fmax(fmax(a, b), fmax(c, d));
    return 0.0;
}

/* MP5 (Sec. 3, the five-point REC of the list of substep steps): the value at i+1/2 from
 * s = (u_{i-2}, ..., u_{i+2}), following Suresh & Huynh (1997).  The unlimited
 * value is the fifth-order point-value Lagrange interpolant at i+1/2, weights
 * (3, -20, 90, 60, -5)/128, since ECHO reconstructs point values.  The
 * monotonicity-preserving bound uses alpha = 4 and eps = 1e-10. */
double orc_mp5(const double *s)
{
    double um2 = s[0], um1 = s[1], u0 = s[2], up1 = s[3], up2 = s[4];
    double uor = (3.0 * um2 - 20.0 * um1 + 90.0 * u0 + 60.0 * up1 - 5.0 * up2) / 128.0;
    double ump = u0 + minmod2(up1 - u0, MP5_ALPHA * (u0 - um1));
    if ((uor - u0) * (uor - ump) <= MP5_EPS) return uor;
    double djm1 = um2 - 2.0 * um1 + u0;
    double dj = um1 - 2.0 * u0 + up1;
    double djp1 = u0 - 2.0 * up1 + up2;
    double dm4p = minmod4(4.0 * dj - djp1, 4.0 * djp1 - dj, dj, djp1);
    double dm4m = minmod4(4.0 * dj - djm1, 4.0 * djm1 - dj, dj, djm1);
    double uul = u0 + MP5_ALPHA * (u0 - um1);
    double uav = 0.5 * (u0 + up1);
    double umd = uav - 0.5 * dm4p;
    double ulc = u0 + 0.5 * (u0 - um1) + 4.0 / 3.0 * dm4m;
    double umin = fmax(fmin(fmin(u0, up1), umd), fmin(fmin(u0, uul), ulc));
    double umax = fmin(fmax(fmax(u0, up1), umd), fmax(fmax(u0, uul), ulc));
    return uor + minmod2(umin - uor, umax - uor);
}

/* Linear reconstruction (Sec. 4, last paragraph: the faster variant uses linear
 * reconstruction instead of MP5; the limiter is not named there).  Monotonized-
 * central slope of cell i from (u_{i-1}, u_i, u_{i+1}):
 * minmod(2 (u_i - u_{i-1}), (u_{i+1} - u_{i-1})/2, 2 (u_{i+1} - u_i)); the value at
 * i+1/2 is u_i + slope/2. */
static double mc_slope(double um1, double u0, double up1)
{
    double a = 2.0 * (u0 - um1), b = 0.5 * (up1 - um1), c = 2.0 * (up1 - u0);
    if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
    if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
    return 0.0;
}

/* value at i+1/2 from s = (u_{i-1}, u_i, u_{i+1}) */
double orc_mc(const double *s) { return s[1] + 0.5 * mc_slope(s[0], s[1], s[2]); }

/* Right-biased MP5 state at i+1/2: the mirror stencil (u_{i+3}, ..., u_{i-1}). */
static double mp5_right(const double *s6)
{
    double m[5] = {s6[5], s6[4], s6[3], s6[2], s6[1]};
    return orc_mp5(m);
}

static double mp5_left(const double *s6) { return orc_mp5(s6); }

/* left and right states at i+1/2 from s6 = (u_{i-2}, ..., u_{i+3}) with the
 * configured reconstruction */
static double rec_left(const orc_cfg *g, const double *s6)
{
    return g->rec == 1 ? orc_mc(s6 + 1) : mp5_left(s6);
}

static double rec_right(const orc_cfg *g, const double *s6)
{
    if (g->rec == 1) {
        double m[3] = {s6[4], s6[3], s6[2]};
        return orc_mc(m);
    }
    return mp5_right(s6);
}

/* INT (Sec. 3 step 1): staggered value to the cell centre along its own direction,
 * from faces (i-3/2, i-1/2, i+1/2, i+3/2) in s.  Second order: mean of the two
 * nearest faces.  High order (HO): the fourth-order midpoint Lagrange interpolant
 * (-1, 9, 9, -1)/16. */
double orc_int(const double *s, int ho)
{
    if (ho) return (-s[0] + 9.0 * s[1] + 9.0 * s[2] - s[3]) / 16.0;
    return 0.5 * (s[1] + s[2]);
}

/* DER (Sec. 3 step 3): derivative at a centre from the six staggered values
 * (i-5/2, ..., i+5/2) in s.  Second order: (F_{i+1/2} - F_{i-1/2})/h.  High order:
 * each staggered value is first corrected as Fc = F - d2F/24 + 3 d4F/640 (d2, d4
 * the central second and fourth differences on the staggered grid), which makes
 * the difference quotient sixth-order accurate. */
static double der_corr(const double *s, int j) /* corrected value at s[j] */
{
    double d2 = s[j - 1] - 2.0 * s[j] + s[j + 1];
    double d4 = s[j - 2] - 4.0 * s[j - 1] + 6.0 * s[j] - 4.0 * s[j + 1] + s[j + 2];
    return s[j] - d2 / 24.0 + 3.0 * d4 / 640.0;
}

double orc_der(const double *s, double h, int ho)
{
    if (!ho) return (s[3] - s[2]) / h;
    /* needs s[-?]: stencil positions 0..5 are i-5/2..i+5/2; corrections at 2 and 3
       use 0..4 and 1..5 */
    return (der_corr(s, 3) - der_corr(s, 2)) / h;
}

/* ------------------------------------------------------------------------- */
/* Conservative-to-primitive inversion (Sec. 3 step 1, "iterative Newton")   */
/* ------------------------------------------------------------------------- */
/* One-dimensional Newton scheme on W = rho h G^2.  With the invariants S^2, B^2,
 * (S.B) and the identity S = (W + B^2) v - (v.B) B (from the definition of S with
 * E = -v x B), the velocity and pressure are functions of W:
 *   v^2(W) = [S^2 W^2 + (S.B)^2 (B^2 + 2W)] / [W^2 (W + B^2)^2],
 *   p(W)   = (gam-1)/gam [W (1 - v^2) - D sqrt(1 - v^2)],
 * and W solves f(W) = W - p + (1 + v^2) B^2/2 - (S.B)^2/(2 W^2) - U = 0.
 * Newton with the analytic derivative; a trial point outside the domain
 * (W <= 0, v^2 >= 1, not finite) halves the step.  The iteration stops after an
 * undamped step with |dW| <= tol W and one more polishing step (after such a step
 * the error is about tol^2 W, and the polishing step squares it again). */

typedef struct { double D, S2, B2, SB, U, gm1g; } c2p_inv;

static double v2_of_w(const c2p_inv *q, double W)
{
    double wb = W + q->B2;
    return (q->S2 * W * W + q->SB * q->SB * (q->B2 + 2.0 * W)) / (W * W * wb * wb);
}

/* f(W) and f'(W) */
static void c2p_fdf(const c2p_inv *q, double W, double *f, double *df)
{
    double v2 = v2_of_w(q, W);
    double wb = W + q->B2;
    double sq1 = sqrt(1.0 - v2);
    double p = q->gm1g * (W * (1.0 - v2) - q->D * sq1);
    double dv2 = -2.0 * q->SB * q->SB / (W * W * W * wb) - 2.0 * v2 / wb;
    double dp = q->gm1g * ((1.0 - v2) - W * dv2 + q->D * dv2 / (2.0 * sq1));
    *f = W - p + 0.5 * (1.0 + v2) * q->B2 - q->SB * q->SB / (2.0 * W * W) - q->U;
    *df = 1.0 - dp + 0.5 * q->B2 * dv2 + q->SB * q->SB / (W * W * W);
}

static int w_ok(const c2p_inv *q, double W)
{
    if (!(W > 0.0) || !isfinite(W)) return 0;
    double v2 = v2_of_w(q, W);
    return isfinite(v2) && v2 < 1.0;
}

static void c2p_setup(const double *u, const double *B, double gam, c2p_inv *q)
{
    q->D = u[0];
    q->S2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    q->B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    q->SB = u[1] * B[0] + u[2] * B[1] + u[3] * B[2];
    q->U = u[4];
    q->gm1g = (gam - 1.0) / gam;
}

/* Exported for the derivative test. */
void orc_c2p_fdf(const double *u, const double *B, double gam, double W,
                 double *f, double *df)
{
    c2p_inv q;
    c2p_setup(u, B, gam, &q);
    c2p_fdf(&q, W, f, df);
}

/* Returns 0 on success, 1 on failure.  prim_out = (rho, vx, vy, vz, p). */
int orc_c2p(const double *u, const double *B, double gam, double W0, double tol,
            int maxit, double *prim_out, double *W_out, int *iters)
{
    c2p_inv q;
    c2p_setup(u, B, gam, &q);
    double W = W0;
    for (int k = 0; k < 64 && !w_ok(&q, W); k++)
        W = (W > 0.0 && isfinite(W)) ? 2.0 * W : fabs(q.U) + 1.0;
    int it = 0, conv = 0, polish = 0;
    while (it < maxit) {
        double f, df;
        c2p_fdf(&q, W, &f, &df);
        double dW = -f / df;
        if (!isfinite(dW)) break;
        double lam = 1.0, Wn = W + dW;
        for (int k = 0; k < 60 && !w_ok(&q, Wn); k++) {
            lam *= 0.5;
            Wn = W + lam * dW;
        }
        it++;
        if (!w_ok(&q, Wn)) break;
        double step = fabs(Wn - W);
        W = Wn;
        if (polish) { conv = 1; break; }
        if (lam == 1.0 && step <= tol * W) polish = 1;
    }
    *iters = it;
    *W_out = W;
    double v2 = v2_of_w(&q, W);
    double sq1 = sqrt(1.0 - v2);
    double lor = 1.0 / sq1;
    double p = q.gm1g * (W * (1.0 - v2) - q.D * sq1);
    double rho = q.D / lor;
    /* v = (S + (S.B) B / W) / (W + B^2) */
    double wb = W + q.B2;
    for (int i = 0; i < 3; i++)
        prim_out[1 + i] = (u[1 + i] + q.SB * B[i] / W) / wb;
    prim_out[0] = rho;
    prim_out[4] = p;
    int ok = conv && isfinite(p) && isfinite(rho) && p > 0.0 && rho > 0.0 && v2 < 1.0;
    return ok ? 0 : 1;
}

/* Batched C2P over n independent states: u[5][n], B[3][n], W0[n] -> prim[5][n],
 * W[n], it[n]; returns the number of failures. */
long orc_c2p_batch(long n, const double *u, const double *B, const double *W0,
                   double gam, double tol, int maxit, double *prim, double *W, int *it)
{
    long fails = 0;
    for (long c = 0; c < n; c++) {
        double uu[5], bb[3], pp[5];
        for (int v = 0; v < 5; v++) uu[v] = u[v * n + c];
        for (int v = 0; v < 3; v++) bb[v] = B[v * n + c];
        fails += orc_c2p(uu, bb, gam, W0[c], tol, maxit, pp, &W[c], &it[c]);
        for (int v = 0; v < 5; v++) prim[v * n + c] = pp[v];
    }
    return fails;
}

/* ------------------------------------------------------------------------- */
/* UCT edge field (Sec. 3 step 4; Eq. 10)                                     */
/* ------------------------------------------------------------------------- */
/* Upwind constrained transport, four-state form (Londrillo & Del Zanna 2004,
 * Del Zanna et al. 2007) for the edge along c at (a+1/2, b+1/2), (a, b, c) cyclic:
 *   vL/vR: the a-face left/right velocity states (components a and b) already
 *          reconstructed along b to the edge, index [s][t] with s the a-side state
 *          and t the b-side state;
 *   Ba[t]: the staggered B_a reconstructed along b (t = L, R);
 *   Bb[s]: the staggered B_b reconstructed along a (s = L, R);
 *   apa/ama, apb/amb: the HLL speeds on the a- and b-faces that meet at the edge.
 * E^{st} = v_b^{st} Ba[t] - v_a^{st} Bb[s];
 * E = sum_{st} w_a(s) w_b(t) E^{st} / ((apa+ama)(apb+amb))
 *     + apa ama (Bb[R] - Bb[L]) / (apa+ama) - apb amb (Ba[R] - Ba[L]) / (apb+amb),
 * with w(L) = a+, w(R) = a-. */
double orc_uct_point(const double va[2][2], const double vb[2][2], const double *Ba,
                     const double *Bb, double apa, double ama, double apb, double amb)
{
    double wa[2] = {apa, ama}, wb[2] = {apb, amb};
    double sa = apa + ama, sb = apb + amb;
    double e4 = 0.0;
    if (sa > 0.0 && sb > 0.0) {
        for (int s = 0; s < 2; s++)
            for (int t = 0; t < 2; t++)
                e4 += wa[s] * wb[t] * (vb[s][t] * Ba[t] - va[s][t] * Bb[s]);
        e4 /= sa * sb;
    } else {
        for (int s = 0; s < 2; s++)
            for (int t = 0; t < 2; t++)
                e4 += 0.25 * (vb[s][t] * Ba[t] - va[s][t] * Bb[s]);
    }
    double da = sa > 0.0 ? apa * ama * (Bb[1] - Bb[0]) / sa : 0.0;
    double db = sb > 0.0 ? apb * amb * (Ba[1] - Ba[0]) / sb : 0.0;
    return e4 + da - db;
}

/* ------------------------------------------------------------------------- */
/* Grid-level steps                                                           */
/* ------------------------------------------------------------------------- */

/* Step 1a: cell-centred field.  UCT: INT of each staggered component along its
 * own direction; otherwise the field is already cell-centred. */
static void cell_field(const orc_cfg *g, const double *bf, double *bc)
{
    long n = ncell(g);
    if (!g->uct) {
        memcpy(bc, bf, 3 * n * sizeof(double));
        return;
    }
#pragma omp parallel for collapse(2)
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++)
                for (int d = 0; d < 3; d++) {
                    const double *b = bf + d * n;
                    /* faces i-3/2, i-1/2, i+1/2, i+3/2 are indices i-2, i-1, i, i+1 */
                    double s[4] = {b[at(g, i, j, k, d, -2)], b[at(g, i, j, k, d, -1)],
                                   b[at(g, i, j, k, d, 0)], b[at(g, i, j, k, d, 1)]};
                    bc[d * n + at(g, i, j, k, d, 0)] = orc_int(s, g->ho);
                }
}

/* Step 1: INT + C2P.  prim[8][n] = rho, vx, vy, vz, p, Bx, By, Bz (cell centres).
 * W holds the previous W (warm guess) on entry and the new W on exit.  guessarr is
 * the caller's guess when g->guess == 2. */
static void int_c2p(const orc_cfg *g, const double *cons, const double *bf, double *W,
                    const double *guessarr, double *prim, int *itc, int *stat)
{
    long n = ncell(g);
    cell_field(g, bf, prim + 5 * n);
#pragma omp parallel for
    for (long c = 0; c < n; c++) {
        double u[5], B[3], p[5], Wn;
        for (int v = 0; v < 5; v++) u[v] = cons[v * n + c];
        for (int v = 0; v < 3; v++) B[v] = prim[(5 + v) * n + c];
        double W0;
        int fb = 0;
        if (g->guess == 1) W0 = u[4];
        else if (g->guess == 2) {
            W0 = guessarr[c];
            c2p_inv q;
            c2p_setup(u, B, g->gam, &q);
            if (!w_ok(&q, W0)) { W0 = W[c]; fb = 1; }
        } else W0 = W[c];
        int it;
        int bad = orc_c2p(u, B, g->gam, W0, g->tol, g->maxit, p, &Wn, &it);
        for (int v = 0; v < 5; v++) prim[v * n + c] = p[v];
        W[c] = Wn;
        itc[c] = it;
        stat[c] = bad | (fb << 1);
    }
}

/* Step 2 at one interface: the left and right reconstructed states (prim 5 +
 * field 3) at the face above cell (i,j,k) along d.  UCT: the normal field is the
 * staggered face value; the other components are MP5 of primitives (rho, v, p and
 * the transverse cell-centred field).  A state with rho <= 0, p <= 0 or v^2 >= 1
 * is replaced by the first-order (cell) value.  Returns the number of such
 * replacements. */
static int face_states(const orc_cfg *g, const double *prim, const double *bf, int d,
                       int i, int j, int k, double *L, double *R)
{
    long n = ncell(g);
    for (int v = 0; v < 8; v++) {
        double s6[6];
        for (int m = 0; m < 6; m++) s6[m] = prim[v * n + at(g, i, j, k, d, m - 2)];
        L[v] = rec_left(g, s6);
        R[v] = rec_right(g, s6);
    }
    if (g->uct) L[5 + d] = R[5 + d] = bf[d * n + at(g, i, j, k, d, 0)];
    int nfb = 0;
    double *st[2] = {L, R};
    for (int q = 0; q < 2; q++) {
        double *x = st[q];
        double v2 = x[1] * x[1] + x[2] * x[2] + x[3] * x[3];
        if (!(x[0] > 0.0) || !(x[4] > 0.0) || !(v2 < 1.0)) {
            long cc = at(g, i, j, k, d, q);  /* cell i for L, i+1 for R */
            for (int v = 0; v < 8; v++) x[v] = prim[v * n + cc];
            if (g->uct) x[5 + d] = bf[d * n + at(g, i, j, k, d, 0)];
            nfb++;
        }
    }
    return nfb;
}

/* Steps 2-3 along direction d: numerical fluxes at every face, then
 * rhs -= DER_d(flux).  UCT face data: velocity states (components d and d+1)
 * and the HLL speeds, kept for step 4.  Returns the max of a+ and a- seen. */
static double sweep(const orc_cfg *g, const double *prim, const double *bf, int d,
                    double *rhs_c, double *rhs_b, double *fvel /*[4][n]*/,
                    double *fap, double *fam, long *recfb)
{
    long n = ncell(g);
    int ncomp = g->uct ? 5 : 8;
    double *flux = malloc(8 * n * sizeof(double));
    int e = (d + 1) % 3;
    long nfb = 0;
#pragma omp parallel for collapse(2) reduction(+ : nfb)
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                double L[8], R[8], fh[8], ap, am;
                nfb += face_states(g, prim, bf, d, i, j, k, L, R);
                orc_hll(L, L + 5, R, R + 5, g->gam, d, fh, &ap, &am);
                long f = at(g, i, j, k, d, 0);
                for (int c = 0; c < 8; c++) flux[c * n + f] = fh[c];
                fap[f] = ap;
                fam[f] = am;
                fvel[0 * n + f] = L[1 + d];
                fvel[1 * n + f] = L[1 + e];
                fvel[2 * n + f] = R[1 + d];
                fvel[3 * n + f] = R[1 + e];
            }
    *recfb += nfb;
    double amax = 0.0;
    for (long f = 0; f < n; f++) amax = fmax(amax, fmax(fap[f], fam[f]));
    double h = hdir(g, d);
#pragma omp parallel for collapse(2)
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                long c0 = at(g, i, j, k, d, 0);
                for (int c = 0; c < ncomp; c++) {
                    double s[6];
                    /* faces i-5/2 .. i+5/2 are face indices i-3 .. i+2 */
                    for (int m = 0; m < 6; m++) s[m] = flux[c * n + at(g, i, j, k, d, m - 3)];
                    double der = orc_der(s, h, g->ho);
                    if (c < 5) rhs_c[c * n + c0] -= der;
                    else rhs_b[(c - 5) * n + c0] -= der;
                }
            }
    free(flux);
    return amax;
}

/* Step 4: edge field along c at every edge, from the a-faces (a = c+1) and the
 * b-faces (b = c+2), using the data each sweep stored. */
static void uct_edges(const orc_cfg *g, const double *bf, int c, double *const *fvel,
                      double *const *fap, double *const *fam, double *E)
{
    long n = ncell(g);
    int a = (c + 1) % 3, b = (c + 2) % 3;
#pragma omp parallel for collapse(2)
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                double va[2][2], vb[2][2], Ba[2], Bb[2], s6[6];
                /* the a-face velocity states along b: fvel[a] holds (v_a, v_b) for the
                   left state in slots 0,1 and the right state in slots 2,3, because
                   b = a+1 cyclically */
                for (int s = 0; s < 2; s++) {
                    for (int m = 0; m < 6; m++)
                        s6[m] = fvel[a][(2 * s + 0) * n + at(g, i, j, k, b, m - 2)];
                    va[s][0] = rec_left(g, s6);
                    va[s][1] = rec_right(g, s6);
                    for (int m = 0; m < 6; m++)
                        s6[m] = fvel[a][(2 * s + 1) * n + at(g, i, j, k, b, m - 2)];
                    vb[s][0] = rec_left(g, s6);
                    vb[s][1] = rec_right(g, s6);
                }
                for (int m = 0; m < 6; m++) s6[m] = bf[a * n + at(g, i, j, k, b, m - 2)];
                Ba[0] = rec_left(g, s6);
                Ba[1] = rec_right(g, s6);
                for (int m = 0; m < 6; m++) s6[m] = bf[b * n + at(g, i, j, k, a, m - 2)];
                Bb[0] = rec_left(g, s6);
                Bb[1] = rec_right(g, s6);
                long e0 = at(g, i, j, k, 0, 0);
                long ea1 = at(g, i, j, k, b, 1); /* a-face one step up along b */
                long eb1 = at(g, i, j, k, a, 1); /* b-face one step up along a */
                double apa = fmax(fap[a][e0], fap[a][ea1]);
                double ama = fmax(fam[a][e0], fam[a][ea1]);
                double apb = fmax(fap[b][e0], fap[b][eb1]);
                double amb = fmax(fam[b][e0], fam[b][eb1]);
                E[e0] = orc_uct_point(va, vb, Ba, Bb, apa, ama, apb, amb);
            }
}

/* Curl of an edge field with DER (Sec. 3, Eq. 10 and step 4):
 * out_a = sign * (D_b E_c - D_c E_b) on the a-faces, (a, b, c) cyclic.
 * sign = -1 gives dB/dt from the electric field; sign = +1 gives B = curl A. */
static void curl_edges(const orc_cfg *g, const double *E, double sign, double *out)
{
    long n = ncell(g);
    for (int a = 0; a < 3; a++) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        double hb = hdir(g, b), hc = hdir(g, c);
#pragma omp parallel for collapse(2)
        for (int k = 0; k < g->nz; k++)
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) {
                    double s[6];
                    /* edges c at b-1/2 and b+1/2 around the face are indices b-1, b */
                    for (int m = 0; m < 6; m++) s[m] = E[c * n + at(g, i, j, k, b, m - 3)];
                    double dbec = orc_der(s, hb, g->ho);
                    for (int m = 0; m < 6; m++) s[m] = E[b * n + at(g, i, j, k, c, m - 3)];
                    double dceb = orc_der(s, hc, g->ho);
                    out[a * n + at(g, i, j, k, 0, 0)] += sign * (dbec - dceb);
                }
    }
}

/* B (faces) += curl A, A given on edges [3][n]. */
void orc_curl_apot(const orc_cfg *g, const double *A, double *bf)
{
    set_threads(g);
    curl_edges(g, A, 1.0, bf);
}

/* Discrete divergence of the face field at cell centres with the same DER. */
void orc_divb(const orc_cfg *g, const double *bf, double *div)
{
    set_threads(g);
    long n = ncell(g);
    memset(div, 0, n * sizeof(double));
    for (int d = 0; d < 3; d++) {
        double h = hdir(g, d);
#pragma omp parallel for collapse(2)
        for (int k = 0; k < g->nz; k++)
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) {
                    double s[6];
                    for (int m = 0; m < 6; m++) s[m] = bf[d * n + at(g, i, j, k, d, m - 3)];
                    div[at(g, i, j, k, 0, 0)] += orc_der(s, h, g->ho);
                }
    }
}

static void stats_add(orc_stats *st, long n, const int *itc, const int *stat)
{
    for (long c = 0; c < n; c++) {
        st->cells++;
        st->iters += itc[c];
        if (itc[c] > st->itmax) st->itmax = itc[c];
        if (stat[c] & 1) st->failures++;
        if (stat[c] & 2) st->fallbacks++;
    }
}

/* The full right-hand side L(U) of Eq. 9-10 for one substep.  cons[5][n] and
 * bf[3][n] are the state; W[n] the warm guess (updated).  Outputs rhs_c[5][n],
 * rhs_b[3][n] and, optionally, prim[8][n] and the largest HLL speed. */
int orc_rhs(const orc_cfg *g, const double *cons, const double *bf, double *W,
            const double *guessarr, double *rhs_c, double *rhs_b, double *prim_out,
            double *amax_out, orc_stats *st)
{
    set_threads(g);
    long n = ncell(g);
    double *prim = prim_out ? prim_out : malloc(8 * n * sizeof(double));
    int *itc = malloc(n * sizeof(int)), *stat = malloc(n * sizeof(int));
    /* step 1 */
    int_c2p(g, cons, bf, W, guessarr, prim, itc, stat);
    long f0 = st->failures;
    stats_add(st, n, itc, stat);
    /* steps 2-3 */
    memset(rhs_c, 0, 5 * n * sizeof(double));
    memset(rhs_b, 0, 3 * n * sizeof(double));
    double *fvel[3], *fap[3], *fam[3];
    double amax = 0.0;
    for (int d = 0; d < 3; d++) {
        fvel[d] = malloc(4 * n * sizeof(double));
        fap[d] = malloc(n * sizeof(double));
        fam[d] = malloc(n * sizeof(double));
        double a = sweep(g, prim, bf, d, rhs_c, rhs_b, fvel[d], fap[d], fam[d],
                         &st->rec_fallbacks);
        amax = fmax(amax, a);
    }
    /* step 4 */
    if (g->uct) {
        double *E = malloc(3 * n * sizeof(double));
        for (int c = 0; c < 3; c++) uct_edges(g, bf, c, fvel, fap, fam, E + c * n);
        curl_edges(g, E, -1.0, rhs_b);
        free(E);
    }
    for (int d = 0; d < 3; d++) { free(fvel[d]); free(fap[d]); free(fam[d]); }
    if (amax_out) *amax_out = amax;
    free(itc);
    free(stat);
    if (!prim_out) free(prim);
    return st->failures > f0 ? 1 : 0;
}

/* Cell-centred primitives and conserved variables from primitives and the field
 * (initialisation, Sec. 2 definitions): W = rho h G^2 is also returned as the
 * first warm guess. */
void orc_set_state(const orc_cfg *g, const double *prim5, const double *bf,
                   double *cons, double *W)
{
    set_threads(g);
    long n = ncell(g);
    double *bc = malloc(3 * n * sizeof(double));
    cell_field(g, bf, bc);
#pragma omp parallel for
    for (long c = 0; c < n; c++) {
        double p[5], B[3], u[5];
        for (int v = 0; v < 5; v++) p[v] = prim5[v * n + c];
        for (int v = 0; v < 3; v++) B[v] = bc[v * n + c];
        orc_prim2cons(p, B, g->gam, u);
        for (int v = 0; v < 5; v++) cons[v * n + c] = u[v];
        double v2 = p[1] * p[1] + p[2] * p[2] + p[3] * p[3];
        W[c] = (p[0] + g->gam / (g->gam - 1.0) * p[4]) / (1.0 - v2);
    }
    free(bc);
}

/* Step 5: one Runge-Kutta step in Shu-Osher form (the paper uses Runge-Kutta
 * substeps, Sec. 3 step 5; the third-order strong-stability-preserving scheme is
 * the default, the second-order one serves the faster variant of Sec. 4):
 *   SSP-RK3: U1 = Un + dt L(Un); U2 = 3/4 Un + 1/4 (U1 + dt L(U1));
 *            U(n+1) = 1/3 Un + 2/3 (U2 + dt L(U2)).
 *   SSP-RK2: U1 = Un + dt L(Un); U(n+1) = 1/2 Un + 1/2 (U1 + dt L(U1)).
 * dt = cfl * min(h) / max(a+, a-) over all faces of the first substep, cut so
 * that t does not pass t_end.  Returns 0, or 1 if any C2P failed. */
int orc_step(const orc_cfg *g, double *cons, double *bf, double *W, const double *guessarr,
             double *t, double t_end, double *dt_out, orc_stats *st)
{
    long n = ncell(g);
    long nc = 5 * n, nb = 3 * n;
    double *u0 = malloc(nc * sizeof(double)), *b0 = malloc(nb * sizeof(double));
    double *rc = malloc(nc * sizeof(double)), *rb = malloc(nb * sizeof(double));
    memcpy(u0, cons, nc * sizeof(double));
    memcpy(b0, bf, nb * sizeof(double));
    int bad = 0;
    double amax;
    bad |= orc_rhs(g, cons, bf, W, guessarr, rc, rb, NULL, &amax, st);
    double hmin = fmin(hdir(g, 0), fmin(hdir(g, 1), hdir(g, 2)));
    double dt = g->cfl * hmin / amax;
    if (*t + dt > t_end) dt = t_end - *t;
    for (long q = 0; q < nc; q++) cons[q] = u0[q] + dt * rc[q];
    for (long q = 0; q < nb; q++) bf[q] = b0[q] + dt * rb[q];
    bad |= orc_rhs(g, cons, bf, W, guessarr, rc, rb, NULL, NULL, st);
    if (g->rk == 2) {
        for (long q = 0; q < nc; q++) cons[q] = 0.5 * u0[q] + 0.5 * (cons[q] + dt * rc[q]);
        for (long q = 0; q < nb; q++) bf[q] = 0.5 * b0[q] + 0.5 * (bf[q] + dt * rb[q]);
    } else {
        for (long q = 0; q < nc; q++) cons[q] = 0.75 * u0[q] + 0.25 * (cons[q] + dt * rc[q]);
        for (long q = 0; q < nb; q++) bf[q] = 0.75 * b0[q] + 0.25 * (bf[q] + dt * rb[q]);
        bad |= orc_rhs(g, cons, bf, W, guessarr, rc, rb, NULL, NULL, st);
        for (long q = 0; q < nc; q++)
            cons[q] = u0[q] / 3.0 + 2.0 / 3.0 * (cons[q] + dt * rc[q]);
        for (long q = 0; q < nb; q++)
            bf[q] = b0[q] / 3.0 + 2.0 / 3.0 * (bf[q] + dt * rb[q]);
    }
    *t += dt;
    if (dt_out) *dt_out = dt;
    free(u0); free(b0); free(rc); free(rb);
    return bad;
}

/* Primitives (rho, v, p) and cell-centred B for output: INT + C2P of the state. */
int orc_primitives(const orc_cfg *g, const double *cons, const double *bf, double *W,
                   double *prim8, orc_stats *st)
{
    set_threads(g);
    long n = ncell(g);
    int *itc = malloc(n * sizeof(int)), *stat = malloc(n * sizeof(int));
    orc_cfg g2 = *g;
    if (g2.guess == 2) g2.guess = 0;
    int_c2p(&g2, cons, bf, W, NULL, prim8, itc, stat);
    long f0 = st->failures;
    stats_add(st, n, itc, stat);
    free(itc);
    free(stat);
    return st->failures > f0 ? 1 : 0;
}

/* Sums of the conserved cell variables and face fields with Neumaier compensated
 * summation: tot[0..4] = D, Sx, Sy, Sz, U; tot[5..7] = face Bx, By, Bz. */
void orc_totals(const orc_cfg *g, const double *cons, const double *bf, double *tot)
{
    long n = ncell(g);
    for (int v = 0; v < 8; v++) {
        const double *a = v < 5 ? cons + v * n : bf + (v - 5) * n;
        double s = 0.0, comp = 0.0;
        for (long c = 0; c < n; c++) {
            double x = a[c], t = s + x;
            if (fabs(s) >= fabs(x)) comp += (s - t) + x;
            else comp += (x - t) + s;
            s = t;
        }
        tot[v] = s + comp;
    }
}
