/*
 * kerr_oracle.c -- plain, slow FP64 CPU oracle for geodesic integration in the
 * Kerr metric (arXiv:1706.07062, "GRay2").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference leg may load it.  It shares no code,
 * header or constant with the CUDA library, and it never reads anything the
 * CUDA path produced.
 *
 * What it computes, and from which passage:
 *   - the Cartesian Kerr-Schild metric g = eta + f l l            (Sec. 2.1, eq. def:CKS, eq. CKSr)
 *   - the Boyer-Lindquist metric                                  (Sec. 2.1, eq. 1)
 *   - metric derivatives by complex-step differentiation (no hand algebra)
 *   - the inverse metric by Gaussian elimination (not eta - f l l)
 *   - the geodesic acceleration from the Christoffel form          (Sec. 2.1, eq. geo)
 *   - classic fixed-step 4th-order Runge-Kutta                     (Sec. 3)
 *   - adaptive step doubling, termination and surface clipping: the paper uses
 *     fixed steps only and states the termination rule in words (Sec. 4: stop
 *     when the photon is close to the horizon or escapes beyond the initial
 *     radius); the controller constants below are this project's reading and
 *     the CUDA path implements the same reading.
 *
 * Deliberately NOT the paper's optimised form (eqs. opt0/opti): the CUDA path
 * uses that form, so the two agree only if both are right.
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Metrics, evaluated in complex arithmetic so that a complex step gives      */
/* exact-to-rounding partial derivatives.  Every operation used is analytic.  */
/* ------------------------------------------------------------------------ */

/* Cartesian Kerr-Schild metric, Sec. 2.1 eq. def:CKS with M = 1:
 *   g_ab = eta_ab + f l_a l_b,
 *   f    = 2 r^3 / (r^4 + a^2 z^2),
 *   l_a  = (1, (r x + a y)/(r^2 + a^2), (r y - a x)/(r^2 + a^2), z / r),
 * where r solves x^2 + y^2 + z^2 = r^2 + a^2 (1 - z^2 / r^2)  (eq. CKSr).
 * The positive root of that quadratic in r^2 is
 *   r^2 = (R^2 - a^2)/2 + sqrt((R^2 - a^2)^2/4 + a^2 z^2).              */
static void ks_metric_c(double a, const cplx X[4], cplx g[4][4])
{
    cplx x = X[1], y = X[2], z = X[3];
    cplx R2 = x * x + y * y + z * z;
    cplx d = R2 - a * a;
    cplx r2 = 0.5 * d + csqrt(0.25 * d * d + a * a * z * z);
    cplx r = csqrt(r2);
    cplx f = 2.0 * r * r2 / (r2 * r2 + a * a * z * z);
    cplx l[4];
    l[0] = 1.0;
    l[1] = (r * x + a * y) / (r2 + a * a);
    l[2] = (r * y - a * x) / (r2 + a * a);
    l[3] = z / r;
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n)
            g[m][n] = f * l[m] * l[n];
    g[0][0] += -1.0;
    g[1][1] += 1.0;
    g[2][2] += 1.0;
    g[3][3] += 1.0;
}

/* Boyer-Lindquist metric, Sec. 2.1 eq. 1 with M = 1, coordinates
 * (t, r, theta, phi):
 *   g_tt = -(1 - 2r/rho^2),  g_tphi = -2 r a sin^2(theta)/rho^2,
 *   g_rr = rho^2/Delta,      g_thth = rho^2,
 *   g_phph = (r^2 + a^2 + 2 r a^2 sin^2(theta)/rho^2) sin^2(theta),
 *   rho^2 = r^2 + a^2 cos^2(theta),  Delta = r^2 - 2r + a^2.            */
static void bl_metric_c(double a, const cplx X[4], cplx g[4][4])
{
    cplx r = X[1], th = X[2];
    cplx s = csin(th), c = ccos(th);
    cplx s2 = s * s;
    cplx rho2 = r * r + a * a * c * c;
    cplx Delta = r * r - 2.0 * r + a * a;
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n)
            g[m][n] = 0.0;
    g[0][0] = -(1.0 - 2.0 * r / rho2);
    g[0][3] = g[3][0] = -2.0 * r * a * s2 / rho2;
    g[1][1] = rho2 / Delta;
    g[2][2] = rho2;
    g[3][3] = (r * r + a * a + 2.0 * r * a * a * s2 / rho2) * s2;
}

typedef void (*metric_fn)(double a, const cplx X[4], cplx g[4][4]);

/* g_{mn} and dg[al][m][n] = d g_{mn} / d x^al, the latter by the complex
 * step  d/dx F(x) = Im F(x + i h) / h  with h = 1e-30 (no subtraction, so the
 * derivative is exact to rounding).                                        */
static void metric_and_derivs(metric_fn m, double a, const double x[4],
                              double g[4][4], double dg[4][4][4])
{
    const double hs = 1e-30;
    cplx X[4], G[4][4];
    for (int i = 0; i < 4; ++i)
        X[i] = x[i];
    m(a, X, G);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            g[i][j] = creal(G[i][j]);
    for (int al = 0; al < 4; ++al) {
        X[al] = x[al] + I * hs;
        m(a, X, G);
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j)
                dg[al][i][j] = cimag(G[i][j]) / hs;
        X[al] = x[al];
    }
}

/* Inverse of a 4x4 matrix by Gauss-Jordan elimination with partial
 * pivoting.  Returns 0 on success, -1 if a pivot vanishes.                 */
static int invert4(const double A[4][4], double B[4][4])
{
    double M[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            M[i][j] = A[i][j];
            M[i][4 + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int c = 0; c < 4; ++c) {
        int p = c;
        for (int i = c + 1; i < 4; ++i)
            if (fabs(M[i][c]) > fabs(M[p][c]))
                p = i;
        if (M[p][c] == 0.0)
            return -1;
        if (p != c)
            for (int j = 0; j < 8; ++j) {
                double t = M[c][j];
                M[c][j] = M[p][j];
                M[p][j] = t;
            }
        double inv = 1.0 / M[c][c];
        for (int j = 0; j < 8; ++j)
            M[c][j] *= inv;
        for (int i = 0; i < 4; ++i)
            if (i != c) {
                double fct = M[i][c];
                for (int j = 0; j < 8; ++j)
                    M[i][j] -= fct * M[c][j];
            }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            B[i][j] = M[i][4 + j];
    return 0;
}

/* Geodesic right-hand side, Sec. 2.1 eq. geo:
 *   d x^mu / d lambda = k^mu,
 *   d k^mu / d lambda = -1/2 g^{mu nu} (g_{nu al,be} + g_{nu be,al} - g_{al be,nu}) k^al k^be.
 * State y = (x^0..x^3, k^0..k^3).                                          */
static void rhs_geo(metric_fn m, double a, const double y[8], double dy[8])
{
    double g[4][4], gi[4][4], dg[4][4][4];
    metric_and_derivs(m, a, y, g, dg);
    if (invert4(g, gi) != 0) {
        for (int i = 0; i < 8; ++i)
            dy[i] = NAN;
        return;
    }
    const double *k = y + 4;
    for (int mu = 0; mu < 4; ++mu) {
        dy[mu] = k[mu];
        double acc = 0.0;
        for (int nu = 0; nu < 4; ++nu) {
            double s = 0.0;
            for (int al = 0; al < 4; ++al)
                for (int be = 0; be < 4; ++be)
                    s += (dg[be][nu][al] + dg[al][nu][be] - dg[nu][al][be]) * k[al] * k[be];
            acc += gi[mu][nu] * s;
        }
        dy[4 + mu] = -0.5 * acc;
    }
}

/* Classic 4th-order Runge-Kutta step (Sec. 3): four RHS evaluations.
 * k1 may be passed in (already evaluated at y) to share it.               */
static void rk4_step(metric_fn m, double a, const double y[8], const double k1in[8],
                     double h, double out[8])
{
    double k1[8], k2[8], k3[8], k4[8], t[8];
    if (k1in)
        memcpy(k1, k1in, sizeof k1);
    else
        rhs_geo(m, a, y, k1);
    for (int i = 0; i < 8; ++i)
        t[i] = y[i] + 0.5 * h * k1[i];
    rhs_geo(m, a, t, k2);
    for (int i = 0; i < 8; ++i)
        t[i] = y[i] + 0.5 * h * k2[i];
    rhs_geo(m, a, t, k3);
    for (int i = 0; i < 8; ++i)
        t[i] = y[i] + h * k3[i];
    rhs_geo(m, a, t, k4);
    for (int i = 0; i < 8; ++i)
        out[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Two classic RK4 steps of h/2 each, starting with the shared k1. */
static void rk4_two_halves(metric_fn m, double a, const double y[8], const double k1[8],
                           double h, double out[8])
{
    double mid[8];
    rk4_step(m, a, y, k1, 0.5 * h, mid);
    rk4_step(m, a, mid, NULL, 0.5 * h, out);
}

/* ------------------------------------------------------------------------ */
/* Public helpers                                                           */
/* ------------------------------------------------------------------------ */

/* Kerr-Schild radius r(x, y, z) from eq. CKSr (real arithmetic). */
double oracle_ks_r(double a, double x, double y, double z)
{
    double d = x * x + y * y + z * z - a * a;
    double r2 = 0.5 * d + sqrt(0.25 * d * d + a * a * z * z);
    return sqrt(r2);
}

/* coords: 0 = Cartesian Kerr-Schild (t,x,y,z), 1 = Boyer-Lindquist (t,r,th,ph) */
static metric_fn pick_metric(int coords) { return coords == 1 ? bl_metric_c : ks_metric_c; }

void oracle_metric(int coords, double a, const double x[4], double g[16])
{
    double G[4][4], dG[4][4][4];
    metric_and_derivs(pick_metric(coords), a, x, G, dG);
    memcpy(g, G, sizeof G);
}

void oracle_metric_derivs(int coords, double a, const double x[4], double dg[64])
{
    double G[4][4], dG[4][4][4];
    metric_and_derivs(pick_metric(coords), a, x, G, dG);
    memcpy(dg, dG, sizeof dG);
}

int oracle_inverse_metric(int coords, double a, const double x[4], double gi[16])
{
    double G[4][4], dG[4][4][4], Gi[4][4];
    metric_and_derivs(pick_metric(coords), a, x, G, dG);
    int rc = invert4(G, Gi);
    memcpy(gi, Gi, sizeof Gi);
    return rc;
}

void oracle_rhs(int coords, double a, const double y[8], double dy[8])
{
    rhs_geo(pick_metric(coords), a, y, dy);
}

/* Fixed-step classic RK4 (Sec. 3), no termination: writes every `stride`-th
 * state (including the initial one) to traj, nsteps/stride + 1 rows of 8.  */
void oracle_rk4_fixed(int coords, double a, const double y0[8], double h,
                      int64_t nsteps, int64_t stride, double *traj)
{
    metric_fn m = pick_metric(coords);
    double y[8], yn[8];
    memcpy(y, y0, sizeof y);
    int64_t row = 0;
    memcpy(traj, y, sizeof y);
    ++row;
    for (int64_t s = 1; s <= nsteps; ++s) {
        rk4_step(m, a, y, NULL, h, yn);
        memcpy(y, yn, sizeof y);
        if (s % stride == 0) {
            memcpy(traj + 8 * row, y, sizeof y);
            ++row;
        }
    }
}

/* g_{mn} k^m k^n with the oracle's metric. */
static double norm2(double a, const double y[8])
{
    double g[4][4], dg[4][4][4];
    metric_and_derivs(ks_metric_c, a, y, g, dg);
    double s = 0.0;
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n)
            s += g[m][n] * y[4 + m] * y[4 + n];
    return s;
}

/* Solve g_{mn} k^m k^n = target for k^t with the spatial k^i held fixed:
 * A kt^2 + B kt + C = 0 with A = g_tt, B = 2 g_ti k^i, C = g_ij k^i k^j - target.
 * branch < 0 picks the smaller root (past-directed), > 0 the larger one,
 * 0 the root nearest the current k^t (keeps the branch when re-normalising
 * inside the ergoregion, where both roots can have the same sign).
 * Returns 0, or -1 when there is no real root.                              */
static int solve_kt(double a, double y[8], double target, int branch)
{
    double g[4][4], dg[4][4][4];
    metric_and_derivs(ks_metric_c, a, y, g, dg);
    double A = g[0][0], B = 0.0, C = -target;
    for (int i = 1; i < 4; ++i) {
        B += 2.0 * g[0][i] * y[4 + i];
        for (int j = 1; j < 4; ++j)
            C += g[i][j] * y[4 + i] * y[4 + j];
    }
    double disc = B * B - 4.0 * A * C;
    if (!(disc >= 0.0) || A == 0.0)
        return -1;
    double q = -0.5 * (B + copysign(sqrt(disc), B));
    double r1 = q / A, r2 = (q != 0.0) ? C / q : r1;
    double lo = fmin(r1, r2), hi = fmax(r1, r2);
    if (branch == 0)
        y[4] = (fabs(lo - y[4]) <= fabs(hi - y[4])) ? lo : hi;
    else
        y[4] = branch < 0 ? lo : hi;
    return 0;
}

/* Camera initial condition (the paper defers its camera to GRay 2013; this
 * is the reading used throughout the project):
 *   observer direction n = (sin i, 0, cos i), image axes e_al = (0,1,0),
 *   e_be = (-cos i, 0, sin i); pixel centres al_p = -w + (p + 1/2) 2w/nx,
 *   be_q = -w + (q + 1/2) 2w/ny; ray index = q nx + p;
 *   start x = r_obs n + al e_al + be e_be, t = 0, spatial k = -n,
 *   k^t from the null condition, past-directed (backward ray tracing).     */
int oracle_camera_ic(double a, double incl, double r_obs, double w, int32_t nx,
                     int32_t ny, int64_t idx, double y0[8])
{
    int64_t p = idx % nx, q = idx / nx;
    double al = -w + (p + 0.5) * 2.0 * w / nx;
    double be = -w + (q + 0.5) * 2.0 * w / ny;
    double si = sin(incl), ci = cos(incl);
    y0[0] = 0.0;
    y0[1] = r_obs * si - be * ci;
    y0[2] = al;
    y0[3] = r_obs * ci + be * si;
    y0[5] = -si;
    y0[6] = 0.0;
    y0[7] = -ci;
    return solve_kt(a, y0, 0.0, -1);
}

/* Particle initial condition: position x^i and coordinate velocity
 * v^i = dx^i/dt; u^i = u^t v^i with u^t from g_{mn} u^m u^n = -1, i.e.
 * u^t = 1/sqrt(-(g_tt + 2 g_ti v^i + g_ij v^i v^j)).  -1 if not time-like. */
int oracle_particle_ic(double a, const double x[4], const double v[3], double y0[8])
{
    double g[4][4], dg[4][4][4];
    metric_and_derivs(ks_metric_c, a, x, g, dg);
    double V[4] = {1.0, v[0], v[1], v[2]};
    double s = 0.0;
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n)
            s += g[m][n] * V[m] * V[n];
    for (int i = 0; i < 4; ++i)
        y0[i] = x[i];
    if (!(s < 0.0))
        return -1;
    double ut = 1.0 / sqrt(-s);
    for (int i = 0; i < 4; ++i)
        y0[4 + i] = ut * V[i];
    return 0;
}

/* Constants of motion at a Cartesian KS state: out = (E, L_z, Q, u^2).
 *   p_m = g_mn k^n, E = -p_t, L_z = x p_y - y p_x  (Killing vectors d_t, d_phi),
 *   p_theta = cot(th) (x p_x + y p_y) - r sin(th) p_z  (theta is shared by the
 *   KS and BL charts), Carter's constant
 *   Q = p_theta^2 + cos^2(th) [a^2 (mu^2 - E^2) + L_z^2 / sin^2(th)],
 *   mu^2 = -u^2, u^2 = k^m p_m.                                            */
void oracle_constants(double a, const double y[8], double out[4])
{
    double g[4][4], dg[4][4][4];
    metric_and_derivs(ks_metric_c, a, y, g, dg);
    double p[4];
    for (int m = 0; m < 4; ++m) {
        p[m] = 0.0;
        for (int n = 0; n < 4; ++n)
            p[m] += g[m][n] * y[4 + n];
    }
    double u2 = 0.0;
    for (int m = 0; m < 4; ++m)
        u2 += p[m] * y[4 + m];
    double E = -p[0];
    double Lz = y[1] * p[2] - y[2] * p[1];
    double r = oracle_ks_r(a, y[1], y[2], y[3]);
    double c = y[3] / r;
    double s2 = 1.0 - c * c;
    double s = sqrt(s2);
    double pth = (c / s) * (y[1] * p[1] + y[2] * p[2]) - r * s * p[3];
    double Q = pth * pth + c * c * (a * a * (-u2 - E * E) + Lz * Lz / s2);
    out[0] = E;
    out[1] = Lz;
    out[2] = Q;
    out[3] = u2;
}

/* ------------------------------------------------------------------------ */
/* Adaptive integration with termination                                    */
/* ------------------------------------------------------------------------ */

enum { ST_ESCAPED = 1, ST_CAPTURED = 2, ST_ENDTIME = 3, ST_MAXSTEPS = 4, ST_NONFINITE = 6 };

typedef struct {
    double tol;          /* error tolerance (rtol = atol = tol)                 */
    double h0;           /* first trial step in lambda                          */
    int64_t max_steps;   /* cap on attempted steps                              */
    double r_escape;     /* > 0: fixed escape radius; == 0: start radius; < 0: none */
    double t_end;        /* stop when t crosses t_end; NaN or inf: none          */
    int32_t renorm_every;/* > 0: every n accepted steps re-solve k^t so that     */
                         /* g k k keeps its initial value; 0: off               */
    int32_t clip_maxit;  /* iterations of the surface root-find                 */
    /* Conditioning test only (0 = off, the plain integration): every accepted
     * step that starts at r >= noise_zone * r_h has each component of its
     * increment y_new - y scaled by (1 + noise * u), u uniform in [-1, 1)
     * drawn per geodesic, step and component -- a model of the rounding that
     * FP32 arithmetic leaves in each step of the FP32+Kahan path outside its
     * FP64 zone.                                                             */
    double noise;
    double noise_zone;
    uint64_t noise_seed;
} oracle_opts;

/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the output function applied to a counter.     */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* Uniform in [-1, 1) from 53 random bits. */
static double uniform_pm1(uint64_t bits) { return (double)(bits >> 11) * 0x1p-52 - 1.0; }

/* Per-geodesic stream of the noise: FNV-1a over the bytes of its start state. */
static uint64_t state_seed(const double y0[8], uint64_t seed)
{
    const unsigned char *p = (const unsigned char *)y0;
    uint64_t h = 1469598103934665603ull ^ seed;
    for (int i = 0; i < 64; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

typedef struct {
    int64_t attempts;
    int64_t accepted;
    int64_t rhs_evals;
} oracle_counts;

static int all_finite(const double y[8])
{
    for (int i = 0; i < 8; ++i)
        if (!isfinite(y[i]))
            return 0;
    return 1;
}

/* One step-doubling attempt of size h from y (k1 = F(y) given):
 * y_full = RK4(y, h), y_half = RK4(RK4(y, h/2), h/2),
 * delta = (y_half - y_full)/15,
 * err = max over the 7 components other than x^0 of
 *       |delta_i| / (tol (1 + max(|y_i|, |y_half_i|))).
 * x^0 is left out because t never enters the right-hand side.              */
static double attempt(metric_fn m, double a, const double y[8], const double k1[8],
                      double h, double tol, double yhalf[8])
{
    double yfull[8];
    rk4_step(m, a, y, k1, h, yfull);
    rk4_two_halves(m, a, y, k1, h, yhalf);
    double err = 0.0;
    for (int i = 1; i < 8; ++i) {
        double d = (yhalf[i] - yfull[i]) / 15.0;
        double sc = tol * (1.0 + fmax(fabs(y[i]), fabs(yhalf[i])));
        double e = fabs(d) / sc;
        if (!(e <= err))       /* NaN propagates into err */
            err = e;
    }
    return err;
}

/* Step-size factor after an attempt: 0.9 err^(-1/5) clamped to [0.2, 5];
 * err == 0 gives 5; a non-finite err gives 0.2.                            */
static double step_factor(double err)
{
    if (!isfinite(err))
        return 0.2;
    if (err == 0.0)
        return 5.0;
    double f = 0.9 * pow(err, -0.2);
    return fmin(5.0, fmax(0.2, f));
}

/* Event function values. */
static double ev_r(double a, const double y[8], double rstop)
{
    return oracle_ks_r(a, y[1], y[2], y[3]) - rstop;
}

/* Clip the accepted step [y_old, y_old -> y_new over h] onto the surface
 * s(y) = 0 with s(y_old) and s(y_new) of opposite sign.  The step as a
 * function of its length, Phi(eta) = two RK4 half steps of eta/2 from y_old
 * (so Phi(h) = y_new), is searched with the Illinois variant of regula falsi
 * until |s| <= stol, the bracket collapses, or maxit iterations.          */
typedef double (*event_fn)(double a, const double y[8], double c);

static double clip(metric_fn m, double a, const double yold[8], const double k1[8],
                   const double ynew[8], double h, event_fn ev, double c, double stol,
                   int maxit, double yout[8], oracle_counts *cnt)
{
    double lo = 0.0, hi = h;
    double slo = ev(a, yold, c), shi = ev(a, ynew, c);
    int side = 0;
    double eta_out = h;
    memcpy(yout, ynew, 8 * sizeof(double));
    for (int it = 0; it < maxit; ++it) {
        double eta = hi - shi * (hi - lo) / (shi - slo);
        if (!(eta > lo && eta < hi))
            eta = 0.5 * (lo + hi);
        double yt[8];
        rk4_two_halves(m, a, yold, k1, eta, yt);
        cnt->rhs_evals += 7;
        double st = ev(a, yt, c);
        memcpy(yout, yt, sizeof yt);
        eta_out = eta;
        if (fabs(st) <= stol)
            break;
        if ((st > 0) == (shi > 0)) {
            hi = eta;
            shi = st;
            if (side == 1)
                slo *= 0.5;
            side = 1;
        } else {
            lo = eta;
            slo = st;
            if (side == -1)
                shi *= 0.5;
            side = -1;
        }
        if (hi - lo <= 1e-15 * h)
            break;
    }
    return eta_out;
}

static double ev_t(double a, const double y[8], double tend)
{
    (void)a;
    return y[0] - tend;
}

static double ev_z(double a, const double y[8], double unused)
{
    (void)a;
    (void)unused;
    return y[3];
}

/* Prograde ISCO radius (Bardeen, Press & Teukolsky 1972), M = 1. */
static double r_isco(double a)
{
    double z1 = 1.0 + cbrt(1.0 - a * a) * (cbrt(1.0 + a) + cbrt(1.0 - a));
    double z2 = sqrt(3.0 * a * a + z1 * z1);
    return 3.0 + z2 - sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
}

/* Equatorial-crossing labels (the surrogate's training targets; the paper
 * has none, this is the project's reading).  A crossing is a step whose
 * end has z of the other sign (or zero); it is located on that step with the
 * same root-find as the clipping, on z = 0.  Recorded: the KS radius and the
 * KS azimuth phi = atan2(y, x) - atan2(a, r) wrapped to (-pi, pi] of the first
 * two crossings, and the redshift of a prograde Keplerian emitter at the
 * first one, g = 1 / (u^t (1 - Omega xi)) with Omega = 1/(r^{3/2} + a),
 * u^t = (r^{3/2} + a) / (r^{3/4} sqrt(r^{3/2} - 3 r^{1/2} + 2a)) and
 * xi = L_z / E of the ray (NaN inside the ISCO).  Missing values are NaN.    */
typedef struct {
    int count;
    double v[5]; /* r1, phi1, r2, phi2, g1 */
} crossings;

static void record_crossing(metric_fn m, double a, const double yold[8], const double k1[8],
                            const double yend[8], double h_used, int maxit, double xi,
                            crossings *cr, oracle_counts *cnt)
{
    const double z0 = yold[3], z1 = yend[3];
    if (cr->count >= 2 || !((z0 > 0 && z1 <= 0) || (z0 < 0 && z1 >= 0)))
        return;
    double yc[8];
    /* z tolerance scaled by the radius at the nearer end of the step */
    const double r0 = oracle_ks_r(a, yold[1], yold[2], yold[3]);
    const double r1 = oracle_ks_r(a, yend[1], yend[2], yend[3]);
    clip(m, a, yold, k1, yend, h_used, ev_z, 0.0, 1e-12 * (1.0 + fmin(r0, r1)), maxit, yc, cnt);
    const double rc = oracle_ks_r(a, yc[1], yc[2], yc[3]);
    double ph = atan2(yc[2], yc[1]) - atan2(a, rc);
    while (ph <= -M_PI)
        ph += 2.0 * M_PI;
    while (ph > M_PI)
        ph -= 2.0 * M_PI;
    cr->v[2 * cr->count] = rc;
    cr->v[2 * cr->count + 1] = ph;
    if (cr->count == 0) {
        if (rc >= r_isco(a)) {
            const double s = sqrt(rc), r32 = rc * s;
            const double ut = (r32 + a) / (sqrt(s) * s * sqrt(r32 - 3.0 * s + 2.0 * a));
            const double Om = 1.0 / (r32 + a);
            cr->v[4] = 1.0 / (ut * (1.0 - Om * xi));
        }
    }
    cr->count++;
}

/* Integrate one geodesic with adaptive step doubling until an event.
 * Termination (the paper's rule of Sec. 4 made precise):
 *   captured : r < 1.01 r_h,  r_h = 1 + sqrt(1 - a^2)
 *   escaped  : r > r_esc and x^i k^i > 0 (moving outward); r_esc is
 *              opts.r_escape if > 0, the start radius if == 0, none if < 0
 *   end time : t - t_end changes sign from its initial value
 *   max steps: attempts reach opts.max_steps
 * Events are tested after each accepted step in the order above; a crossing
 * step is clipped onto the surface.  A start inside 1.01 r_h is "captured"
 * with no step.  Returns the status.                                        */
int oracle_trace_one(double a, const double y0[8], const oracle_opts *o, double yend[8],
                     oracle_counts *cnt, double cross_out[5])
{
    metric_fn m = ks_metric_c;
    memset(cnt, 0, sizeof *cnt);
    memcpy(yend, y0, 8 * sizeof(double));
    crossings cr;
    cr.count = 0;
    for (int i = 0; i < 5; ++i)
        cr.v[i] = NAN;
    if (cross_out)
        memcpy(cross_out, cr.v, sizeof cr.v);
    if (!all_finite(y0))
        return ST_NONFINITE;
    const double rh = 1.0 + sqrt(1.0 - a * a);
    const double rcap = 1.01 * rh;
    const double r0 = oracle_ks_r(a, y0[1], y0[2], y0[3]);
    const double resc = o->r_escape > 0 ? o->r_escape : (o->r_escape == 0 ? r0 : INFINITY);
    const int use_t = isfinite(o->t_end);
    const double s0t = y0[0] - o->t_end;
    const double u2_0 = norm2(a, y0);
    double c0[4];
    oracle_constants(a, y0, c0);
    const double xi = c0[1] / c0[0];
    if (r0 < rcap)
        return ST_CAPTURED;

    double y[8], k1[8], yh[8], ye[8];
    memcpy(y, y0, sizeof y);
    double h = o->h0;
    int64_t since_renorm = 0;
    const uint64_t nseed = o->noise > 0.0 ? state_seed(y0, o->noise_seed) : 0;
    const double noise_r = o->noise_zone * rh;
    int status = ST_MAXSTEPS;
    for (;;) {
        if (cnt->attempts >= o->max_steps) {
            status = ST_MAXSTEPS;
            break;
        }
        cnt->attempts++;
        rhs_geo(m, a, y, k1);
        double err = attempt(m, a, y, k1, h, o->tol, yh);
        cnt->rhs_evals += 11;
        double fac = step_factor(err);
        if (!(err <= 1.0)) {
            h *= fac;
            continue;
        }
        cnt->accepted++;
        if (o->noise > 0.0 && oracle_ks_r(a, y[1], y[2], y[3]) >= noise_r) {
            for (int i = 0; i < 8; ++i) {
                const uint64_t ctr = nseed + 8u * (uint64_t)cnt->accepted + (uint64_t)i;
                yh[i] = y[i] + (yh[i] - y[i]) * (1.0 + o->noise * uniform_pm1(splitmix64(ctr)));
            }
        }
        if (!all_finite(yh)) {
            memcpy(y, yh, sizeof y);
            status = ST_NONFINITE;
            break;
        }
        /* termination (with the clipped end point ye and its step length) */
        int st = 0;
        double h_used = h;
        memcpy(ye, yh, sizeof ye);
        double rn = oracle_ks_r(a, yh[1], yh[2], yh[3]);
        if (rn < rcap) {
            h_used = clip(m, a, y, k1, yh, h, ev_r, rcap, 1e-12 * rcap, o->clip_maxit, ye, cnt);
            st = ST_CAPTURED;
        } else if (rn > resc && (yh[1] * yh[5] + yh[2] * yh[6] + yh[3] * yh[7]) > 0.0) {
            double rold = oracle_ks_r(a, y[1], y[2], y[3]);
            if (rold <= resc)
                h_used = clip(m, a, y, k1, yh, h, ev_r, resc, 1e-12 * resc, o->clip_maxit, ye,
                              cnt);
            st = ST_ESCAPED;
        } else if (use_t && ((yh[0] - o->t_end > 0) != (s0t > 0))) {
            h_used = clip(m, a, y, k1, yh, h, ev_t, o->t_end,
                          1e-12 * fmax(1.0, fabs(o->t_end)), o->clip_maxit, ye, cnt);
            st = ST_ENDTIME;
        }
        if (cross_out)
            record_crossing(m, a, y, k1, ye, h_used, o->clip_maxit, xi, &cr, cnt);
        memcpy(y, ye, sizeof y);
        if (st) {
            status = st;
            break;
        }
        if (o->renorm_every > 0 && ++since_renorm >= o->renorm_every) {
            since_renorm = 0;
            solve_kt(a, y, u2_0, 0);
        }
        h *= fac;
    }
    memcpy(yend, y, sizeof y);
    if (cross_out)
        memcpy(cross_out, cr.v, sizeof cr.v);
    return status;
}

/* Batch driver: n geodesics (rows of 8, AoS), each with its own spin, spread
 * over nthreads host threads with a shared counter.                        */
typedef struct {
    int64_t n;
    const double *a;
    const double *t_end;   /* per-geodesic end times or NULL */
    const double *y0;
    const oracle_opts *o;
    double *yend;
    int32_t *status;
    int64_t *attempts;
    int64_t *rhs_evals;
    double *cross;         /* n x 5 or NULL */
    int64_t next;
    pthread_mutex_t mu;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *J = (batch_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t i = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (i >= J->n)
            break;
        oracle_counts c;
        oracle_opts o = *J->o;
        if (J->t_end)
            o.t_end = J->t_end[i];
        J->status[i] = oracle_trace_one(J->a[i], J->y0 + 8 * i, &o, J->yend + 8 * i, &c,
                                        J->cross ? J->cross + 5 * i : NULL);
        if (J->attempts)
            J->attempts[i] = c.attempts;
        if (J->rhs_evals)
            J->rhs_evals[i] = c.rhs_evals;
    }
    return NULL;
}

int oracle_trace_batch(int64_t n, const double *a, const double *t_end, const double *y0,
                       const oracle_opts *o, double *yend, int32_t *status, int64_t *attempts,
                       int64_t *rhs_evals, double *cross, int nthreads)
{
    batch_job J = {n, a, t_end, y0, o, yend, status, attempts, rhs_evals, cross, 0,
                   PTHREAD_MUTEX_INITIALIZER};
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 256)
        nthreads = 256;
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t)
        pthread_create(&th[t], NULL, batch_worker, &J);
    for (int t = 0; t < nthreads; ++t)
        pthread_join(th[t], NULL);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Coordinate-time integration (Sec. 2.2, eq. geo_t)                        */
/* ------------------------------------------------------------------------ */

/* With the coordinate time t as the independent variable the state is
 * w = (x, y, z, v^x, v^y, v^z), v = dx/dt.  Along a geodesic k = k^t u with
 * u = (1, v); the affine acceleration A(k) = dk/dlambda is quadratic in k and
 * d/dlambda = k^t d/dt, so
 *   dx^i/dt = v^i,   dv^i/dt = (A^i(k) - v^i A^t(k)) / (k^t)^2
 *                            = A^i(u) - v^i A^t(u).
 * The oracle evaluates A(u) with the Christoffel form (rhs_geo).  (Eq. geo_t
 * writes the same right-hand side in the split-metric variables.)          */
static void rhs_coordtime(metric_fn m, double a, double t, const double w[6], double dw[6])
{
    const double y[8] = {t, w[0], w[1], w[2], 1.0, w[3], w[4], w[5]};
    double dy[8];
    rhs_geo(m, a, y, dy);
    for (int i = 0; i < 3; ++i) {
        dw[i] = w[3 + i];
        dw[3 + i] = dy[5 + i] - w[3 + i] * dy[4];
    }
}

/* Classic RK4 step of the coordinate-time system (Sec. 3). */
static void rk4_step_t(metric_fn m, double a, double t, const double w[6], double h,
                       double out[6])
{
    double k1[6], k2[6], k3[6], k4[6], s[6];
    rhs_coordtime(m, a, t, w, k1);
    for (int i = 0; i < 6; ++i)
        s[i] = w[i] + 0.5 * h * k1[i];
    rhs_coordtime(m, a, t + 0.5 * h, s, k2);
    for (int i = 0; i < 6; ++i)
        s[i] = w[i] + 0.5 * h * k2[i];
    rhs_coordtime(m, a, t + 0.5 * h, s, k3);
    for (int i = 0; i < 6; ++i)
        s[i] = w[i] + h * k3[i];
    rhs_coordtime(m, a, t + h, s, k4);
    for (int i = 0; i < 6; ++i)
        out[i] = w[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Adaptive integration in coordinate time from (t0, w0) to t_end, with the
 * affine integrator's controller (step doubling, err over the six
 * components, the same factor rule).  A trial step never passes t_end: the
 * last accepted step lands on it exactly.  Termination after each accepted
 * step: captured r < 1.01 r_h; escaped r > r_esc while moving outward in the
 * direction of integration (sign(t_end - t0) x.v > 0); end time reached.
 * No surface clipping (the end time needs none).  Returns the status.      */
int oracle_trace_coordtime(double a, double t0, const double w0[6], double t_end,
                           const oracle_opts *o, double wend[6], double *t_out,
                           int64_t *attempts_out)
{
    metric_fn m = ks_metric_c;
    double w[6], t = t0;
    memcpy(w, w0, sizeof w);
    int64_t att = 0;
    int st = 0;
    const double rh = 1.0 + sqrt(fmax(0.0, 1.0 - a * a));
    const double rcap = 1.01 * rh;
    const double r0 = oracle_ks_r(a, w[0], w[1], w[2]);
    const double resc = o->r_escape > 0.0 ? o->r_escape : (o->r_escape == 0.0 ? r0 : INFINITY);
    const double dir = t_end >= t0 ? 1.0 : -1.0;
    double h = dir * o->h0;
    int finite = 1;
    for (int i = 0; i < 6; ++i)
        finite = finite && isfinite(w[i]);
    if (!finite || !isfinite(t0) || !isfinite(t_end))
        st = ST_NONFINITE;
    else if (r0 < rcap)
        st = ST_CAPTURED;
    else if (t_end == t0)
        st = ST_ENDTIME;
    while (st == 0) {
        if (att >= o->max_steps) {
            st = ST_MAXSTEPS;
            break;
        }
        const int last = dir * (t + h - t_end) >= 0.0;   /* this trial reaches t_end */
        const double hs = last ? t_end - t : h;
        ++att;
        double wf[6], wm[6], wh[6];
        rk4_step_t(m, a, t, w, hs, wf);
        rk4_step_t(m, a, t, w, 0.5 * hs, wm);
        rk4_step_t(m, a, t + 0.5 * hs, wm, 0.5 * hs, wh);
        double err = 0.0;
        for (int i = 0; i < 6; ++i) {
            const double d = (wh[i] - wf[i]) / 15.0;
            const double sc = o->tol * (1.0 + fmax(fabs(w[i]), fabs(wh[i])));
            const double e = fabs(d) / sc;
            if (!(e <= err))
                err = e;
        }
        const double fac = step_factor(err);
        if (!(err <= 1.0)) {
            h = hs * fac;
            continue;
        }
        memcpy(w, wh, sizeof w);
        t = last ? t_end : t + hs;
        finite = 1;
        for (int i = 0; i < 6; ++i)
            finite = finite && isfinite(w[i]);
        if (!finite) {
            st = ST_NONFINITE;
            break;
        }
        const double r = oracle_ks_r(a, w[0], w[1], w[2]);
        if (r < rcap)
            st = ST_CAPTURED;
        else if (r > resc && dir * (w[0] * w[3] + w[1] * w[4] + w[2] * w[5]) > 0.0)
            st = ST_ESCAPED;
        else if (last)
            st = ST_ENDTIME;
        h = (last ? h : hs) * fac;
    }
    memcpy(wend, w, sizeof w);
    *t_out = t;
    *attempts_out = att;
    return st;
}
