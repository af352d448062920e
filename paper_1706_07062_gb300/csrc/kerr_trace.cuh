// kerr_trace.cuh -- persistent geodesic-integration kernel.
//
// One geodesic per thread with its whole state in registers.  Threads pull
// geodesic indices from one global counter with warp-aggregated atomics: the
// lanes of a warp that have no geodesic (a ballot) are refilled together by
// a single atomicAdd, so a warp keeps all lanes busy while geodesics of very
// different length (captured, escaping, grazing the photon ring, multi-orbit
// particles) retire at different times.
//
// Per attempted step (arXiv:1706.07062 Sec. 3 classic RK4; the step control
// is this library's): one RK4 step of h and two of h/2 from the same state,
// 11 right-hand sides (Sec. 2.1, eqs. opt0/opti, in kerr_math.cuh).
#pragma once

#include <type_traits>

#include "kerr_math.cuh"

namespace kerr {

enum : int {
    ST_NONE = 0,
    ST_ESCAPED = 1,
    ST_CAPTURED = 2,
    ST_ENDTIME = 3,
    ST_MAXSTEPS = 4,
    ST_TIMEOUT = 5,
    ST_NONFINITE = 6,
    ST_INVALID_IC = 7
};

enum : int { MODE_RAYS = 0, MODE_CAMERA = 1, MODE_PARTICLES = 2 };

// Camera as the kernel sees it: the public kerr_camera plus the index of its
// first ray.
struct CamDev {
    double a, incl, r_obs, w;
    int32_t nx, ny;
    int64_t offset;
};

// Counter slots in the statistics buffer (unsigned long long each).
enum : int {
    SC_GEODESICS = 0,
    SC_ATTEMPTS = 1,
    SC_ACCEPTED = 2,
    SC_RHS32 = 3,
    SC_RHS64 = 4,
    SC_ATT64 = 5,
    SC_STATUS = 8,   // 8 slots: geodesics per status code
    SC_COUNT = 16
};

struct TraceParams {
    int mode;
    int64_t n;
    double a;                   // spin for MODE_RAYS / MODE_PARTICLES
    const double *x0;           // [4][n]
    const double *k0;           // [4][n] (rays) or [3][n] velocities (particles)
    const double *t_end_each;   // [n] per-geodesic end times, or null
    const CamDev *cams;
    int32_t ncam;
    double *x_out, *k_out;      // [4][n]
    int32_t *status, *steps;    // [n]
    float *diag;                // [4][n] or null
    double tol, h0;
    int64_t max_steps;
    double r_escape, t_end, fp64_zone;
    int32_t renorm_every, clip_maxit;
    uint64_t budget_ns;
    unsigned long long *head;   // work-queue counter, zero at launch
    unsigned long long *stats;  // SC_COUNT counters, zero at launch
};

// Per-geodesic constants fixed at set-up.
struct RayConst {
    double a;
    double rcap;     // 1.01 r_h
    double resc;     // escape radius (inf: none)
    double zone_r;   // FP64 zone radius (FP32 path)
    double tend;     // end time (only if use_t)
    double u2_0;     // initial g k k (renormalisation target)
    int use_t;
    int tpos;        // initial sign of t - t_end
};

// ---------------------------------------------------------------------------
// Runge-Kutta pieces
// ---------------------------------------------------------------------------

// Increments d = y(lambda + h) - y(lambda) of one classic RK4 step (Sec. 3)
// from y, with A0 = accel(y) already known: 3 right-hand sides.
template <typename T>
__device__ __forceinline__ void rk4_incr(const T a, const T a2, const T y[8], const T A0[4],
                                         const T h, T d[8])
{
    const T hh = T(0.5) * h;
    T Sk[4], SA[4];
    T m[4], A[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        Sk[j] = y[4 + j];
        SA[j] = A0[j];
        m[j] = k_fma(hh, A0[j], y[4 + j]);
    }
    accel(a, a2, k_fma(hh, y[5], y[1]), k_fma(hh, y[6], y[2]), k_fma(hh, y[7], y[3]), m[0], m[1],
          m[2], m[3], A[0], A[1], A[2], A[3]);
    T m3[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        Sk[j] = k_fma(T(2), m[j], Sk[j]);
        SA[j] = k_fma(T(2), A[j], SA[j]);
        m3[j] = k_fma(hh, A[j], y[4 + j]);
    }
    accel(a, a2, k_fma(hh, m[1], y[1]), k_fma(hh, m[2], y[2]), k_fma(hh, m[3], y[3]), m3[0], m3[1],
          m3[2], m3[3], A[0], A[1], A[2], A[3]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        Sk[j] = k_fma(T(2), m3[j], Sk[j]);
        SA[j] = k_fma(T(2), A[j], SA[j]);
        m[j] = k_fma(h, A[j], y[4 + j]);
    }
    accel(a, a2, k_fma(h, m3[1], y[1]), k_fma(h, m3[2], y[2]), k_fma(h, m3[3], y[3]), m[0], m[1],
          m[2], m[3], A[0], A[1], A[2], A[3]);
    const T h6 = h * T(1.0 / 6.0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        d[j] = h6 * (Sk[j] + m[j]);
        d[4 + j] = h6 * (SA[j] + A[j]);
    }
}

// Two RK4 steps of h/2 from y (A0 = accel(y)): total increment d, 7 RHS.
template <typename T>
__device__ __forceinline__ void two_halves(const T a, const T a2, const T y[8], const T A0[4],
                                           const T h, T d[8])
{
    T d1[8];
    rk4_incr(a, a2, y, A0, T(0.5) * h, d1);
    T ym[8], Am[4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        ym[i] = y[i] + d1[i];
    accel(a, a2, ym[1], ym[2], ym[3], ym[4], ym[5], ym[6], ym[7], Am[0], Am[1], Am[2], Am[3]);
    rk4_incr(a, a2, ym, Am, T(0.5) * h, d);
#pragma unroll
    for (int i = 0; i < 8; ++i)
        d[i] = d1[i] + d[i];
}

// One step-doubling attempt: returns the error measure and the increment of
// the two-half-step solution (10 RHS beyond A0).
template <typename T>
__device__ __forceinline__ T attempt(const T a, const T a2, const T y[8], const T A0[4], const T h,
                                     const T tol, T d[8])
{
    T df[8];
    rk4_incr(a, a2, y, A0, h, df);
    two_halves(a, a2, y, A0, h, d);
    T err = T(0);
#pragma unroll
    for (int i = 1; i < 8; ++i) {
        const T delta = (d[i] - df[i]) * T(1.0 / 15.0);
        const T sc = tol * (T(1) + fmax(fabs(y[i]), fabs(y[i] + d[i])));
        const T e = fabs(delta) / sc;
        err = (e <= err) ? err : e;    // NaN propagates
    }
    return err;
}

template <typename T>
__device__ __forceinline__ T step_factor(T err)
{
    if (!isfinite(err))
        return T(0.2);
    if (err == T(0))
        return T(5);
    const T f = T(0.9) * pow(err, T(-0.2));
    return fmin(T(5), fmax(T(0.2), f));
}

template <bool KAHAN, typename T>
__device__ __forceinline__ void add_incr(T &y, T &c, T d)
{
    if (KAHAN) {
        const T s = d + c;
        const T t = y + s;
        c = s - (t - y);
        y = t;
    } else {
        y = y + d;
    }
}

// Event value on a state (y, c): r - target (kind 0) or t - target (kind 1).
template <bool KAHAN, typename T>
__device__ __forceinline__ T event_value(int kind, T a2, const T y[8], const T c[8], T target)
{
    if (kind == 0)
        return ks_r(a2, y[1], y[2], y[3]) - target;
    return KAHAN ? (y[0] - target) + c[0] : y[0] - target;
}

// Clip an accepted step onto an event surface (Illinois regula falsi on the
// step length eta in (0, h), Phi(eta) = two RK4 half steps from the last
// accepted state).  (y, c) is the last accepted state; on return it holds the
// end point.  Bracket values s_lo = s(y_old) and s_hi = s(y_new).
template <bool KAHAN, typename T>
__device__ void clip(const T a, const T a2, T y[8], T c[8], const T A0[4], const T h, int kind,
                     T target, T s_lo, T s_hi, T stol, T eps, int maxit, uint32_t &nrhs)
{
    T lo = T(0), hi = h;
    int side = 0;
    T ye[8], ce[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        ye[i] = y[i];
        ce[i] = c[i];
    }
    T d[8];
    for (int it = 0; it < maxit; ++it) {
        T eta = hi - s_hi * (hi - lo) / (s_hi - s_lo);
        if (!(eta > lo && eta < hi))
            eta = T(0.5) * (lo + hi);
        two_halves(a, a2, y, A0, eta, d);
        nrhs += 7;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            ye[i] = y[i];
            ce[i] = c[i];
            add_incr<KAHAN>(ye[i], ce[i], d[i]);
        }
        const T s = event_value<KAHAN>(kind, a2, ye, ce, target);
        if (fabs(s) <= stol)
            break;
        if ((s > T(0)) == (s_hi > T(0))) {
            hi = eta;
            s_hi = s;
            if (side == 1)
                s_lo *= T(0.5);
            side = 1;
        } else {
            lo = eta;
            s_lo = s;
            if (side == -1)
                s_hi *= T(0.5);
            side = -1;
        }
        if (hi - lo <= eps * h)
            break;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        y[i] = ye[i];
        c[i] = ce[i];
    }
}

template <typename T> struct Prec;
template <> struct Prec<float> {
    static constexpr float stol = 2e-6f;
    static constexpr float eps = 1e-7f;
};
template <> struct Prec<double> {
    static constexpr double stol = 1e-12;
    static constexpr double eps = 1e-15;
};

// One attempted step with events.  (y, c) is the lane state; h the trial
// step; rn receives r of the new state when a step is accepted.  Returns a
// status code when the geodesic terminates, ST_NONE otherwise.
template <bool KAHAN, typename T>
__device__ __forceinline__ int step_once(const RayConst &rc, const TraceParams &P, T y[8], T c[8],
                                         T &h, T &rn, uint32_t &nrhs, uint32_t &nacc,
                                         int &since_renorm)
{
    const T a = (T)rc.a;
    const T a2 = a * a;
    T A0[4];
    accel(a, a2, y[1], y[2], y[3], y[4], y[5], y[6], y[7], A0[0], A0[1], A0[2], A0[3]);
    T d[8];
    const T err = attempt(a, a2, y, A0, h, (T)P.tol, d);
    nrhs += 11;
    const T fac = step_factor(err);
    if (!(err <= T(1))) {
        h *= fac;
        return ST_NONE;
    }
    ++nacc;
    T yn[8], cn[8];
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        yn[i] = y[i];
        cn[i] = c[i];
        add_incr<KAHAN>(yn[i], cn[i], d[i]);
        finite = finite && isfinite(yn[i]);
    }
    if (!finite) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            y[i] = yn[i];
            c[i] = cn[i];
        }
        return ST_NONFINITE;
    }
    rn = ks_r(a2, yn[1], yn[2], yn[3]);
    const T rcap = (T)rc.rcap;
    const int maxit = P.clip_maxit;
    if (rn < rcap) {
        const T s_lo = event_value<KAHAN>(0, a2, y, c, rcap);
        clip<KAHAN>(a, a2, y, c, A0, h, 0, rcap, s_lo, rn - rcap, Prec<T>::stol * rcap,
                    Prec<T>::eps, maxit, nrhs);
        return ST_CAPTURED;
    }
    const T resc = (T)rc.resc;
    if (rn > resc && k_fma(yn[1], yn[5], k_fma(yn[2], yn[6], yn[3] * yn[7])) > T(0)) {
        const T s_lo = event_value<KAHAN>(0, a2, y, c, resc);
        if (s_lo <= T(0)) {
            clip<KAHAN>(a, a2, y, c, A0, h, 0, resc, s_lo, rn - resc, Prec<T>::stol * resc,
                        Prec<T>::eps, maxit, nrhs);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                y[i] = yn[i];
                c[i] = cn[i];
            }
        }
        return ST_ESCAPED;
    }
    if (rc.use_t) {
        const T tend = (T)rc.tend;
        const T s_hi = event_value<KAHAN>(1, a2, yn, cn, tend);
        if ((s_hi > T(0)) != (rc.tpos != 0)) {
            const T s_lo = event_value<KAHAN>(1, a2, y, c, tend);
            const T sc = fmax(T(1), fabs(tend));
            clip<KAHAN>(a, a2, y, c, A0, h, 1, tend, s_lo, s_hi, Prec<T>::stol * sc, Prec<T>::eps,
                        maxit, nrhs);
            return ST_ENDTIME;
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        y[i] = yn[i];
        c[i] = cn[i];
    }
    if (P.renorm_every > 0 && ++since_renorm >= P.renorm_every) {
        since_renorm = 0;
        double k[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            k[j] = (double)y[4 + j] + (KAHAN ? (double)c[4 + j] : 0.0);
        const KSPoint p = ks_point(rc.a, (double)y[1] + (KAHAN ? (double)c[1] : 0.0),
                                   (double)y[2] + (KAHAN ? (double)c[2] : 0.0),
                                   (double)y[3] + (KAHAN ? (double)c[3] : 0.0));
        if (solve_kt(p, k, rc.u2_0, 0)) {
            y[4] = (T)k[0];
            c[4] = KAHAN ? (T)(k[0] - (double)y[4]) : T(0);
        }
    }
    h *= fac;
    return ST_NONE;
}

// ---------------------------------------------------------------------------
// Set-up and output
// ---------------------------------------------------------------------------

// Builds the FP64 initial state of geodesic `id`; returns ST_NONE when it has
// to be integrated, or the status it ends with right away.
__device__ __forceinline__ int init_geodesic(const TraceParams &P, int64_t id, double y[8],
                                             RayConst &rc)
{
    const int64_t n = P.n;
    double a = P.a;
    int st = ST_NONE;
    if (P.mode == MODE_CAMERA) {
        int lo = 0, hi = P.ncam - 1;
        while (lo < hi) {   // last camera with offset <= id
            const int mid = (lo + hi + 1) >> 1;
            if (P.cams[mid].offset <= id)
                lo = mid;
            else
                hi = mid - 1;
        }
        const CamDev cam = P.cams[lo];
        a = cam.a;
        const int64_t local = id - cam.offset;
        const int64_t p = local % cam.nx, q = local / cam.nx;
        const double al = -cam.w + (p + 0.5) * 2.0 * cam.w / cam.nx;
        const double be = -cam.w + (q + 0.5) * 2.0 * cam.w / cam.ny;
        double si, ci;
        sincos(cam.incl, &si, &ci);
        y[0] = 0.0;
        y[1] = cam.r_obs * si - be * ci;
        y[2] = al;
        y[3] = cam.r_obs * ci + be * si;
        y[5] = -si;
        y[6] = 0.0;
        y[7] = -ci;
        y[4] = 0.0;
        const KSPoint kp = ks_point(a, y[1], y[2], y[3]);
        if (!solve_kt(kp, y + 4, 0.0, -1))
            st = ST_INVALID_IC;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            y[j] = P.x0[j * n + id];
        if (P.mode == MODE_RAYS) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                y[4 + j] = P.k0[j * n + id];
        } else {
            const double v1 = P.k0[id], v2 = P.k0[n + id], v3 = P.k0[2 * n + id];
            const KSPoint kp = ks_point(a, y[1], y[2], y[3]);
            const double lv = 1.0 + kp.lx * v1 + kp.ly * v2 + kp.lz * v3;
            const double s = -1.0 + v1 * v1 + v2 * v2 + v3 * v3 + kp.f * lv * lv;
            if (s < 0.0) {
                const double ut = 1.0 / sqrt(-s);
                y[4] = ut;
                y[5] = ut * v1;
                y[6] = ut * v2;
                y[7] = ut * v3;
            } else {
                // not time-like (or not finite): report the start event, k = 0
                y[4] = y[5] = y[6] = y[7] = 0.0;
                st = isfinite(s) ? ST_INVALID_IC : ST_NONFINITE;
            }
        }
    }
    rc.a = a;
    const double rh = 1.0 + sqrt(fmax(0.0, 1.0 - a * a));
    rc.rcap = 1.01 * rh;
    rc.zone_r = P.fp64_zone * rh;
    const double tend = P.t_end_each ? P.t_end_each[id] : P.t_end;
    rc.use_t = isfinite(tend) ? 1 : 0;
    rc.tend = tend;
    rc.tpos = (y[0] - tend) > 0.0 ? 1 : 0;
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        finite = finite && isfinite(y[i]);
    if (st == ST_NONE && !finite)
        st = ST_NONFINITE;
    const double r0 = finite ? ks_r(a * a, y[1], y[2], y[3]) : 0.0;
    rc.resc = P.r_escape > 0.0 ? P.r_escape : (P.r_escape == 0.0 ? r0 : INFINITY);
    if (st == ST_NONE) {
        const KSPoint kp = ks_point(a, y[1], y[2], y[3]);
        rc.u2_0 = norm2(kp, y + 4);
        if (r0 < rc.rcap)
            st = ST_CAPTURED;
    }
    return st;
}

__device__ __forceinline__ void write_out(const TraceParams &P, int64_t id, const double y[8],
                                          int st, uint32_t nsteps, double a)
{
    const int64_t n = P.n;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        P.x_out[j * n + id] = y[j];
        P.k_out[j * n + id] = y[4 + j];
    }
    P.status[id] = st;
    P.steps[id] = (int32_t)nsteps;
    if (P.diag) {
        float c[4];
        if (st == ST_INVALID_IC || st == ST_NONFINITE) {
            c[0] = c[1] = c[2] = c[3] = __int_as_float(0x7fc00000);
        } else {
            constants(a, y, c);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            P.diag[j * n + id] = c[j];
    }
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One attempted step of an FP32+Kahan geodesic taken in FP64 (inside the
// zone r < fp64_zone r_h, where f l l is large): the compensated pair is
// folded into one FP64 state, stepped, and split back.  Kept out of line so
// that its FP64 registers do not raise the register count of the FP32 loop;
// it only runs for the few steps near the horizon.  The lane state travels
// by value so that the caller's arrays stay in registers.
struct LaneF {
    float y[8], c[8];
    float h, rnow;
};
struct ZoneResult {
    LaneF s;
    int st;
    uint32_t nrhs, nacc;
    int since_renorm;
};

__device__ __noinline__ ZoneResult zone_step(const RayConst rc, const TraceParams &P, LaneF s,
                                             int since_renorm)
{
    double yd[8], cd[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        yd[i] = (double)s.y[i] + (double)s.c[i];
        cd[i] = 0.0;
    }
    double hd = (double)s.h, rd = (double)s.rnow;
    ZoneResult R;
    R.nrhs = 0;
    R.nacc = 0;
    R.st = step_once<false, double>(rc, P, yd, cd, hd, rd, R.nrhs, R.nacc, since_renorm);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        R.s.y[i] = (float)yd[i];
        R.s.c[i] = (float)(yd[i] - (double)R.s.y[i]);
    }
    R.s.h = (float)hd;
    R.s.rnow = (float)rd;
    R.since_renorm = since_renorm;
    return R;
}

// ---------------------------------------------------------------------------
// The persistent kernel.  F32 selects the FP32+Kahan path (with FP64 steps
// inside the zone); otherwise every step is FP64.
// ---------------------------------------------------------------------------
template <bool F32, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) trace_kernel(const TraceParams P)
{
    using T = typename std::conditional<F32, float, double>::type;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;

    bool has = false;
    bool drained = false;
    bool timed_out = false;
    int64_t id = 0;
    RayConst rc;
    T y[8], c[8];
    T h = T(0), rnow = T(0);
    uint32_t nsteps = 0;
    int since_renorm = 0;
    uint32_t c_geo = 0, c_att = 0, c_acc = 0, c_rhs32 = 0, c_rhs64 = 0, c_att64 = 0;
    uint32_t c_st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const unsigned long long t_start = global_ns();
    uint32_t iter = 0;

    for (;;) {
        // ---- refill idle lanes from the queue (one atomic per warp)
        const unsigned need = __ballot_sync(FULL, !has);
        if (need && !drained) {
            const int leader = __ffs(need) - 1;
            const unsigned cnt = __popc(need);
            unsigned long long base = 0;
            if (lane == leader)
                base = atomicAdd(P.head, (unsigned long long)cnt);
            base = __shfl_sync(FULL, base, leader);
            if (base + cnt >= (unsigned long long)P.n)
                drained = true;
            if (!has) {
                const unsigned long long my = base + __popc(need & lt_mask);
                if (my < (unsigned long long)P.n) {
                    id = (int64_t)my;
                    double yd[8];
                    const int st0 = init_geodesic(P, id, yd, rc);
                    ++c_geo;
                    if (st0 != ST_NONE || timed_out) {
                        const int st = st0 != ST_NONE ? st0 : ST_TIMEOUT;
                        write_out(P, id, yd, st, 0, rc.a);
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            c_st[j] += (st == j) ? 1u : 0u;
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            y[i] = (T)yd[i];
                            c[i] = F32 ? (T)(yd[i] - (double)y[i]) : T(0);
                        }
                        h = (T)P.h0;
                        rnow = (T)ks_r(rc.a * rc.a, yd[1], yd[2], yd[3]);
                        nsteps = 0;
                        since_renorm = 0;
                        has = true;
                    }
                }
            }
        }
        if (!__any_sync(FULL, has)) {
            if (drained)      // warp-uniform: derived from the shuffled base
                break;
            continue;
        }
        if (has) {
            int st = ST_NONE;
            if (timed_out) {
                st = ST_TIMEOUT;
            } else if ((int64_t)nsteps >= P.max_steps) {
                st = ST_MAXSTEPS;
            } else {
                ++nsteps;
                ++c_att;
                if (F32 && (double)rnow < rc.zone_r) {
                    LaneF ls;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        ls.y[i] = (float)y[i];
                        ls.c[i] = (float)c[i];
                    }
                    ls.h = (float)h;
                    ls.rnow = (float)rnow;
                    const ZoneResult R = zone_step(rc, P, ls, since_renorm);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        y[i] = (T)R.s.y[i];
                        c[i] = (T)R.s.c[i];
                    }
                    h = (T)R.s.h;
                    rnow = (T)R.s.rnow;
                    since_renorm = R.since_renorm;
                    st = R.st;
                    c_rhs64 += R.nrhs;
                    c_acc += R.nacc;
                    ++c_att64;
                } else {
                    uint32_t r = 0;
                    st = step_once<F32, T>(rc, P, y, c, h, rnow, r, c_acc, since_renorm);
                    if (F32)
                        c_rhs32 += r;
                    else
                        c_rhs64 += r;
                    if (!F32)
                        ++c_att64;
                }
            }
            if (st != ST_NONE) {
                double yd[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    yd[i] = F32 ? (double)y[i] + (double)c[i] : (double)y[i];
                write_out(P, id, yd, st, nsteps, rc.a);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    c_st[j] += (st == j) ? 1u : 0u;
                has = false;
            }
        }
        // ---- wall-time budget (warp-uniform decision)
        if (P.budget_ns && ((++iter & 31u) == 0) && !timed_out) {
            bool over = false;
            if (lane == 0)
                over = (global_ns() - t_start) > P.budget_ns;
            timed_out = __shfl_sync(FULL, over, 0);
        }
    }

    // ---- statistics: warp reduction, one atomic per counter per warp
    auto wsum = [&](uint32_t v) -> unsigned long long {
        unsigned long long s = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(FULL, s, o);
        return s;
    };
    unsigned long long s_geo = wsum(c_geo), s_att = wsum(c_att), s_acc = wsum(c_acc);
    unsigned long long s_r32 = wsum(c_rhs32), s_r64 = wsum(c_rhs64), s_a64 = wsum(c_att64);
    unsigned long long s_st[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        s_st[j] = wsum(c_st[j]);
    if (lane == 0) {
        atomicAdd(P.stats + SC_GEODESICS, s_geo);
        atomicAdd(P.stats + SC_ATTEMPTS, s_att);
        atomicAdd(P.stats + SC_ACCEPTED, s_acc);
        atomicAdd(P.stats + SC_RHS32, s_r32);
        atomicAdd(P.stats + SC_RHS64, s_r64);
        atomicAdd(P.stats + SC_ATT64, s_a64);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            atomicAdd(P.stats + SC_STATUS + j, s_st[j]);
    }
}

} // namespace kerr
