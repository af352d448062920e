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
#include "kerr_df.cuh"

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

enum : int { MODE_RAYS = 0, MODE_CAMERA = 1, MODE_PARTICLES = 2, MODE_POINTS = 3 };

// Camera as the kernel sees it: the public kerr_camera (the inclination as
// its sine and cosine, evaluated once on the host) plus the index of its
// first ray.
struct CamDev {
    double a, sin_incl, cos_incl, r_obs, w;
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
    SC_DEFERRED = 6, // geodesics handed to the zone phase
    SC_REQUEUED = 7, // zone phase: geodesics put back behind waiting ones
    SC_STATUS = 8,   // 8 slots: geodesics per status code; slot 0 (no status)
                     // counts zone-queue hand-overs that timed out (never expected)
    SC_RHS32_ZONE = 16,  // zone phase: FP32 right-hand sides (steps outside the zone)
    SC_ATT32_ZONE = 17,  // zone phase: FP32 attempts
    SC_CLIPS = 18,       // end points clipped onto an event surface
    SC_CLIP_RHS = 19,    // right-hand sides of those clips
    SC_COUNT = 20
};

// State of one geodesic handed from the FP32 phase to the FP64-zone phase
// (96 bytes): the compensated FP32 state and the stepping bookkeeping; the
// per-geodesic constants stay in the constants planes.
struct ZoneEntry {
    float y[8], c[8];
    int64_t id;
    float h, rnow;
    uint32_t nsteps;
    int32_t since_renorm;
    uint32_t seq;      // zone queue: (index + 1) mod 2^32 once written, 0 once read
    int32_t fmt;       // ZE_PAIR: (y, c) is the compensated FP32 pair; ZE_FP64:
                       // the FP64 state, low words in y, high words in c
};
enum : int32_t { ZE_PAIR = 0, ZE_FP64 = 1 };
static_assert(sizeof(ZoneEntry) == 96, "zone entry layout");

// Per-geodesic constants of the FP32 path, one float plane each.
enum : int {
    KC_A = 0,       // spin
    KC_RCAP = 1,    // capture radius 1.01 r_h (rounded from FP64)
    KC_RESC = 2,    // escape radius (inf: none)
    KC_ZONE = 3,    // FP64-zone radius
    KC_TEND = 4,    // end time, high part (float pair)
    KC_TENDLO = 5,  // end time, low part
    KC_U2 = 6,      // initial g k k (renormalisation target)
    KC_FLAGS = 7,   // bit 0: end time in use; bit 1: initial sign of t - t_end
    KC_XI = 8,      // L_z / E of the start state (redshift label)
    KC_COUNT = 9
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
    const int64_t *index;       // camera mode: pixel index of geodesic id (or null: id itself)
    const unsigned long long *n_dev;  // number of geodesics on the device (or null: n)
    const double *points;       // MODE_POINTS: [n][4] (alpha, beta, a, incl)
    double r_obs;               // MODE_POINTS: observer distance
    double *x_out, *k_out;      // [4][n]
    int32_t *status, *steps;    // [n]
    float *diag;                // [4][n] or null
    float *cross;               // [5][n] equatorial-crossing labels or null
    double tol, h0;
    int64_t max_steps;
    double r_escape, t_end, fp64_zone;
    int32_t renorm_every, clip_maxit;
    int32_t zone_df;            // FP32 path: zone steps in float-float (1) or FP64 (0)
    int32_t zone_quantum;       // zone phase: warp iterations between re-queue
                                // points (0: each geodesic runs to its end)
    uint64_t budget_ns;
    const int32_t *abort;       // host-writable stop flag (mapped pinned memory), or null
    unsigned long long *head;   // work-queue counter, zero at launch
    unsigned long long *stats;  // SC_COUNT counters, zero at launch
    float *s_state;             // FP32 path: [16][n] planes y[0..7], c[0..7]
    float *s_const;             // FP32 path: [KC_COUNT][n] planes
    ZoneEntry *zbuf;            // deferred zone geodesics (FP32 path), or null
    int64_t zcap;               // capacity of zbuf
    unsigned long long *zcount; // entries appended, zero at launch
    unsigned long long *zhead;  // zone-phase work-queue counter, zero at launch
    unsigned long long *zpush;  // zone phase: re-queued geodesics, zero at launch
    unsigned long long *zdone;  // zone phase: geodesics finished, zero at launch
    double *traj;               // FP64 path: stored solution [n][traj_cap][9] (lambda, y)
    int32_t traj_cap;           // records per geodesic (the start state is the first)
    int32_t *traj_count;        // [n] records stored
    // FP32 path, deferred clipping (all null: clip in place).  A geodesic whose
    // accepted step crosses an event surface keeps its state from before the
    // step in s_state, the step length in clip_h and the event value at the
    // unclipped end in clip_shi, and is queued in clipq: geodesics whose last
    // step ran in FP32 from the front (count *cq32), those whose last step
    // ran in the zone's arithmetic from the back (count *cq64).
    float *clip_h;              // [n]
    double *clip_shi;           // [n]
    int64_t *clipq;             // [n]
    unsigned long long *cq32, *cq64;
};

// Coordinate-time integration (Sec. 2.2, eq. geo_t): launch parameters.
struct CoordParams {
    int64_t n;
    double a;
    const double *x0;           // [4][n] start events (t, x, y, z)
    const double *v0;           // [3][n] coordinate velocities dx^i/dt
    const double *t_end_each;   // [n] end times, or null: t_end
    double t_end;
    double *x_out;              // [4][n] end events
    double *v_out;              // [3][n] end velocities
    int32_t *status, *steps;    // [n]
    double tol, h0, r_escape;
    int64_t max_steps;
    unsigned long long *head;   // work-queue counter, zero at launch
    unsigned long long *stats;  // SC_COUNT counters, zero at launch
};

#ifndef KERR_TYPES_ONLY

// Per-geodesic constants fixed at set-up.
struct RayConst {
    double a;
    double rcap;     // 1.01 r_h
    double resc;     // escape radius (inf: none)
    double zone_r;   // FP64 zone radius (FP32 path)
    double tend;     // end time (only if use_t)
    double u2_0;     // initial g k k (renormalisation target)
    double xi;       // L_z / E of the start state
    int use_t;
    int tpos;        // initial sign of t - t_end
    // FP32 copies, so that the FP32 loop issues no FP64 conversions;
    // t_end is an unevaluated float pair (tendf + tendlo) to keep the end-time
    // event exact to ~1e-14 relative
    float af, rcapf, rescf, zonef, tendf, tendlo;
    float alo, rcaplo;   // low parts of a and rcap (float-float zone steps)
};

__device__ __forceinline__ void finish_const(RayConst &rc)
{
    rc.af = (float)rc.a;
    rc.rcapf = (float)rc.rcap;
    rc.rescf = (float)rc.resc;
    rc.zonef = (float)rc.zone_r;
    rc.tendf = (float)rc.tend;
    rc.tendlo = isfinite(rc.tend) ? (float)(rc.tend - (double)rc.tendf) : 0.0f;
    rc.alo = (float)(rc.a - (double)rc.af);
    rc.rcaplo = (float)(rc.rcap - (double)rc.rcapf);
}

// Per-precision view of the ray constants.
template <typename T> struct RC;
template <> struct RC<float> {
    static __device__ __forceinline__ float a(const RayConst &r) { return r.af; }
    static __device__ __forceinline__ float rcap(const RayConst &r) { return r.rcapf; }
    static __device__ __forceinline__ float resc(const RayConst &r) { return r.rescf; }
    static __device__ __forceinline__ float tend(const RayConst &r) { return r.tendf; }
    static __device__ __forceinline__ float tendlo(const RayConst &r) { return r.tendlo; }
};
template <> struct RC<dfloat> {
    static __device__ __forceinline__ dfloat a(const RayConst &r) { return dfloat(r.af, r.alo); }
    static __device__ __forceinline__ dfloat rcap(const RayConst &r)
    {
        return dfloat(r.rcapf, r.rcaplo);
    }
    static __device__ __forceinline__ dfloat resc(const RayConst &r) { return dfloat(r.rescf, 0.f); }
    static __device__ __forceinline__ dfloat tend(const RayConst &r)
    {
        return quick_two_sum(r.tendf, r.tendlo);
    }
    static __device__ __forceinline__ dfloat tendlo(const RayConst &) { return dfloat(0.f, 0.f); }
};
template <> struct RC<double> {
    static __device__ __forceinline__ double a(const RayConst &r) { return r.a; }
    static __device__ __forceinline__ double rcap(const RayConst &r) { return r.rcap; }
    static __device__ __forceinline__ double resc(const RayConst &r) { return r.resc; }
    static __device__ __forceinline__ double tend(const RayConst &r) { return r.tend; }
    static __device__ __forceinline__ double tendlo(const RayConst &) { return 0.0; }
};

// ---------------------------------------------------------------------------
// Runge-Kutta pieces
// ---------------------------------------------------------------------------

// How an attempt evaluates its right-hand sides: inline (the compiler
// schedules all of them together), one out-of-line copy (far less code for
// the instruction cache; FP32 and FP64), or out-of-line pairs of independent
// right-hand sides (FP64; float-float is always inline).  The source
// arithmetic of every right-hand side is the same in all three.
enum : int { RHS_INLINE = 0, RHS_CALL = 1, RHS_PAIR = 2 };

template <int RM, typename T>
__device__ __forceinline__ void rhs(const T a, const T a2, const T x, const T y, const T z,
                                    const T kt, const T kx, const T ky, const T kz, T A[4])
{
    if constexpr (RM != RHS_INLINE) {
        const Acc<T> r = accel_call<T>(a, a2, x, y, z, kt, kx, ky, kz);
        A[0] = r.t;
        A[1] = r.x;
        A[2] = r.y;
        A[3] = r.z;
    } else {
        accel(a, a2, x, y, z, kt, kx, ky, kz, A[0], A[1], A[2], A[3]);
    }
}

// Two independent right-hand sides at p and q = (x, y, z, k^t, k^x, k^y, k^z).
template <int RM, typename T>
__device__ __forceinline__ void rhs2(const T a, const T a2, const T p[7], const T q[7], T Ap[4],
                                     T Aq[4])
{
    if constexpr (RM == RHS_PAIR && std::is_same<T, double>::value) {
        const Acc64x2 r = accel_pair(a, a2, p[0], p[1], p[2], p[3], p[4], p[5], p[6], q[0], q[1],
                                     q[2], q[3], q[4], q[5], q[6]);
        Ap[0] = r.p.t;
        Ap[1] = r.p.x;
        Ap[2] = r.p.y;
        Ap[3] = r.p.z;
        Aq[0] = r.q.t;
        Aq[1] = r.q.x;
        Aq[2] = r.q.y;
        Aq[3] = r.q.z;
    } else {
        rhs<RM>(a, a2, p[0], p[1], p[2], p[3], p[4], p[5], p[6], Ap);
        rhs<RM>(a, a2, q[0], q[1], q[2], q[3], q[4], q[5], q[6], Aq);
    }
}

// The final product of an RK4 increment.  FP64: an explicit IEEE multiply,
// which the compiler never fuses into a later addition or subtraction (the
// error measure's d - df, the update y + d), so an increment has the same
// value wherever it is consumed -- in the lane that computed it or, in the
// zone phase's two-lane attempts, in another lane.  Other types: a * b.
template <typename T> __device__ __forceinline__ T k_mul_x(T a, T b) { return a * b; }
__device__ __forceinline__ double k_mul_x(double a, double b) { return __dmul_rn(a, b); }

// Increments d = y(lambda + h) - y(lambda) of one classic RK4 step (Sec. 3)
// from y, with A0 = accel(y) already known: 3 right-hand sides.
template <int RM, typename T>
__device__ __forceinline__ void rk4_incr_body(const T a, const T a2, const T y[8], const T A0[4],
                                              const T h, T d[8])
{
    const T hh = T(0.5) * h;
    if constexpr (!std::is_same<T, dfloat>::value) {
        // With stage momenta m2 = k + (h/2) A0, m3 = k + (h/2) A1 and
        // m4 = k + h A2, the position increment (h/6)(k + 2 m2 + 2 m3 + m4)
        // is h k + (h^2/6)(A0 + A1 + A2), and the momentum increment
        // (h/6)(A0 + 2 (A1 + A2) + A3): three instructions fewer per step
        // than the running stage sums (float-float keeps those).
        T m[4], A[4], C[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            m[j] = k_fma(hh, A0[j], y[4 + j]);
        rhs<RM>(a, a2, k_fma(hh, y[5], y[1]), k_fma(hh, y[6], y[2]), k_fma(hh, y[7], y[3]), m[0],
                m[1], m[2], m[3], A);
        T m3[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            C[j] = A[j];
            m3[j] = k_fma(hh, A[j], y[4 + j]);
        }
        rhs<RM>(a, a2, k_fma(hh, m[1], y[1]), k_fma(hh, m[2], y[2]), k_fma(hh, m[3], y[3]), m3[0],
                m3[1], m3[2], m3[3], A);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            C[j] = C[j] + A[j];
            m[j] = k_fma(h, A[j], y[4 + j]);
        }
        rhs<RM>(a, a2, k_fma(h, m3[1], y[1]), k_fma(h, m3[2], y[2]), k_fma(h, m3[3], y[3]), m[0],
                m[1], m[2], m[3], A);
        const T h6 = h * T(1.0 / 6.0);
        const T hh6 = h * h6;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            d[j] = k_fma(hh6, A0[j] + C[j], h * y[4 + j]);
            d[4 + j] = k_mul_x(h6, k_fma(T(2), C[j], A0[j]) + A[j]);
        }
    } else {
        T Sk[4], SA[4];
        T m[4], A[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            Sk[j] = y[4 + j];
            SA[j] = A0[j];
            m[j] = k_fma(hh, A0[j], y[4 + j]);
        }
        rhs<RM>(a, a2, k_fma(hh, y[5], y[1]), k_fma(hh, y[6], y[2]), k_fma(hh, y[7], y[3]), m[0],
                m[1], m[2], m[3], A);
        T m3[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            Sk[j] = k_fma(T(2), m[j], Sk[j]);
            SA[j] = k_fma(T(2), A[j], SA[j]);
            m3[j] = k_fma(hh, A[j], y[4 + j]);
        }
        rhs<RM>(a, a2, k_fma(hh, m[1], y[1]), k_fma(hh, m[2], y[2]), k_fma(hh, m[3], y[3]), m3[0],
                m3[1], m3[2], m3[3], A);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            Sk[j] = k_fma(T(2), m3[j], Sk[j]);
            SA[j] = k_fma(T(2), A[j], SA[j]);
            m[j] = k_fma(h, A[j], y[4 + j]);
        }
        rhs<RM>(a, a2, k_fma(h, m3[1], y[1]), k_fma(h, m3[2], y[2]), k_fma(h, m3[3], y[3]), m[0],
                m[1], m[2], m[3], A);
        const T h6 = h * T(1.0 / 6.0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            d[j] = k_mul_x(h6, Sk[j] + m[j]);
            d[4 + j] = k_mul_x(h6, SA[j] + A[j]);
        }
    }
}

template <typename T> struct Incr8 {
    T v[8];
};

// One out-of-line copy of the RK4 step for float-float: each float-float
// operation expands to several FP32 instructions, and with every step inlined
// the attempt's code no longer fits the instruction cache (warps then stall
// on instruction fetch).  y[0] (t) does not enter the step.
template <typename T>
static __device__ __noinline__ Incr8<T> rk4_incr_call(const T a, const T a2, const T y1,
                                                      const T y2, const T y3, const T y4,
                                                      const T y5, const T y6, const T y7,
                                                      const T A00, const T A01, const T A02,
                                                      const T A03, const T h)
{
    const T y[8] = {T(0), y1, y2, y3, y4, y5, y6, y7};
    const T A0[4] = {A00, A01, A02, A03};
    Incr8<T> r;
    rk4_incr_body<RHS_CALL>(a, a2, y, A0, h, r.v);
    return r;
}

// RK4 increments: inline, or (float-float with out-of-line right-hand sides)
// through the one out-of-line copy above.
template <int RM = RHS_INLINE, typename T>
__device__ __forceinline__ void rk4_incr(const T a, const T a2, const T y[8], const T A0[4],
                                         const T h, T d[8])
{
    if constexpr (RM == RHS_CALL && std::is_same<T, dfloat>::value) {
        const Incr8<T> r = rk4_incr_call<T>(a, a2, y[1], y[2], y[3], y[4], y[5], y[6], y[7],
                                            A0[0], A0[1], A0[2], A0[3], h);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            d[i] = r.v[i];
    } else {
        rk4_incr_body<RM>(a, a2, y, A0, h, d);
    }
}

// Two RK4 steps from the same y and A0, of lengths h1 and h2, in lockstep:
// their right-hand sides go in pairs.  Each chain's arithmetic is that of
// rk4_incr.
template <int RM, typename T>
__device__ __forceinline__ void rk4_incr2(const T a, const T a2, const T y[8], const T A0[4],
                                          const T h1, const T h2, T d1[8], T d2[8])
{
    if constexpr (!std::is_same<T, double>::value) {
        // other types: the two steps one after the other
        rk4_incr<RM>(a, a2, y, A0, h1, d1);
        rk4_incr<RM>(a, a2, y, A0, h2, d2);
        return;
    }
    const T hh1 = T(0.5) * h1, hh2 = T(0.5) * h2;
    T m1[4], m2[4], A1[4], A2[4], C1[4], C2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        m1[j] = k_fma(hh1, A0[j], y[4 + j]);
        m2[j] = k_fma(hh2, A0[j], y[4 + j]);
    }
    {
        const T p[7] = {k_fma(hh1, y[5], y[1]), k_fma(hh1, y[6], y[2]), k_fma(hh1, y[7], y[3]),
                        m1[0], m1[1], m1[2], m1[3]};
        const T q[7] = {k_fma(hh2, y[5], y[1]), k_fma(hh2, y[6], y[2]), k_fma(hh2, y[7], y[3]),
                        m2[0], m2[1], m2[2], m2[3]};
        rhs2<RM>(a, a2, p, q, A1, A2);
    }
    T n1[4], n2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        C1[j] = A1[j];
        n1[j] = k_fma(hh1, A1[j], y[4 + j]);
        C2[j] = A2[j];
        n2[j] = k_fma(hh2, A2[j], y[4 + j]);
    }
    {
        const T p[7] = {k_fma(hh1, m1[1], y[1]), k_fma(hh1, m1[2], y[2]), k_fma(hh1, m1[3], y[3]),
                        n1[0], n1[1], n1[2], n1[3]};
        const T q[7] = {k_fma(hh2, m2[1], y[1]), k_fma(hh2, m2[2], y[2]), k_fma(hh2, m2[3], y[3]),
                        n2[0], n2[1], n2[2], n2[3]};
        rhs2<RM>(a, a2, p, q, A1, A2);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        C1[j] = C1[j] + A1[j];
        m1[j] = k_fma(h1, A1[j], y[4 + j]);
        C2[j] = C2[j] + A2[j];
        m2[j] = k_fma(h2, A2[j], y[4 + j]);
    }
    {
        const T p[7] = {k_fma(h1, n1[1], y[1]), k_fma(h1, n1[2], y[2]), k_fma(h1, n1[3], y[3]),
                        m1[0], m1[1], m1[2], m1[3]};
        const T q[7] = {k_fma(h2, n2[1], y[1]), k_fma(h2, n2[2], y[2]), k_fma(h2, n2[3], y[3]),
                        m2[0], m2[1], m2[2], m2[3]};
        rhs2<RM>(a, a2, p, q, A1, A2);
    }
    const T h61 = h1 * T(1.0 / 6.0), h62 = h2 * T(1.0 / 6.0);
    const T hh61 = h1 * h61, hh62 = h2 * h62;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        d1[j] = k_fma(hh61, A0[j] + C1[j], h1 * y[4 + j]);
        d1[4 + j] = k_mul_x(h61, k_fma(T(2), C1[j], A0[j]) + A1[j]);
        d2[j] = k_fma(hh62, A0[j] + C2[j], h2 * y[4 + j]);
        d2[4 + j] = k_mul_x(h62, k_fma(T(2), C2[j], A0[j]) + A2[j]);
    }
}

// Two RK4 steps of h/2 from y (A0 = accel(y)): total increment d, 7 RHS.
template <int RM = RHS_INLINE, typename T>
__device__ __forceinline__ void two_halves(const T a, const T a2, const T y[8], const T A0[4],
                                           const T h, T d[8])
{
    T d1[8];
    rk4_incr<RM>(a, a2, y, A0, T(0.5) * h, d1);
    T ym[8], Am[4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        ym[i] = y[i] + d1[i];
    rhs<RM>(a, a2, ym[1], ym[2], ym[3], ym[4], ym[5], ym[6], ym[7], Am);
    rk4_incr<RM>(a, a2, ym, Am, T(0.5) * h, d);
#pragma unroll
    for (int i = 0; i < 8; ++i)
        d[i] = d1[i] + d[i];
}

// Error measure of an FP32 step-doubling attempt: the largest over the
// components i >= 1 of |d_i - df_i| / 15 relative to tol (1 + max(|y_i|,
// |y_i + d_i|)), with d the two-half-step and df the full-step increment
// (Richardson's estimate of the local error of the more accurate solution).
// The running maximum is kept as one fraction num / den: each candidate
// e_i / sc_i is compared by cross-multiplying (sc_i, den > 0, products far
// from overflow), and one division by den remains at the end instead of one
// per component; 1/15 and tol are folded into the scale, |d_i - df_i|
// against 15 tol (1 + max(...)) (one FMA for the scale, no multiply for the
// difference).  A NaN component makes the measure NaN (a rejected step).
__device__ __forceinline__ float err_norm_f(const float y[8], const float d[8], const float df[8],
                                            const float tol)
{
    const float s15 = 15.f * tol;
    float num = 0.f, den = 1.f;
    bool bad = false;
#pragma unroll
    for (int i = 1; i < 8; ++i) {
        const float e = fabsf(d[i] - df[i]);
        const float sc = k_fma(fmaxf(fabsf(y[i]), fabsf(y[i] + d[i])), s15, s15);
        const bool take = e * den > num * sc;
        num = take ? e : num;
        den = take ? sc : den;
        bad = bad || !(e == e);
    }
    return bad ? __int_as_float(0x7fc00000) : __fdiv_rn(num, den);
}

// The same error measure for FP64 and float-float: the max over i of
// |delta_i| / sc_i is kept as one fraction num / den, each comparison
// cross-multiplied (sc_i, den > 0) and one reciprocal at the end instead of a
// division per component.
template <typename T>
__device__ __forceinline__ T err_norm_d(const T y[8], const T d[8], const T df[8], const T tol)
{
    T num = T(0), den = T(1);
#pragma unroll
    for (int i = 1; i < 8; ++i) {
        const T delta = (d[i] - df[i]) * T(1.0 / 15.0);
        const T sc = tol * (T(1) + k_absmax(y[i], y[i] + d[i]));
        const T e = fabs(delta);
        const bool take = !(e * den <= num * sc);
        num = take ? e : num;
        den = take ? sc : den;
    }
    return num * k_rcp(den);
}

// The same measure for the FP64 zone steps of the FP32+Kahan path: 1/15 and
// tol folded into the scale, |d - df| against 15 tol (1 + max(|y|, |y + d|))
// (one FMA for the scale, no multiply for delta): two FP64 instructions fewer
// per component.  It rounds differently from err_norm_d in the last bits,
// which only moves the next trial step by as much; the FP64 path keeps
// err_norm_d.
__device__ __forceinline__ double err_norm_zone(const double y[8], const double d[8],
                                                const double df[8], const double tol)
{
    const double s15 = 15.0 * tol;
    double num = 0.0, den = 1.0;
#pragma unroll
    for (int i = 1; i < 8; ++i) {
        const double e = fabs(d[i] - df[i]);
        const double sc = k_fma(k_absmax(y[i], y[i] + d[i]), s15, s15);
        const bool take = !(e * den <= num * sc);
        num = take ? e : num;
        den = take ? sc : den;
    }
    return num * k_rcp(den);
}

// One step-doubling attempt: returns the error measure and the increment of
// the two-half-step solution (10 RHS beyond A0).  With paired right-hand
// sides the full step and the first half step run in lockstep.
template <int RM = RHS_INLINE, bool ZONE_NORM = false, typename T>
__device__ __forceinline__ T attempt(const T a, const T a2, const T y[8], const T A0[4], const T h,
                                     const T tol, T d[8])
{
    T df[8];
    if constexpr (RM == RHS_PAIR) {
        T d1[8];
        rk4_incr2<RM>(a, a2, y, A0, h, T(0.5) * h, df, d1);
        T ym[8], Am[4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            ym[i] = y[i] + d1[i];
        rhs<RM>(a, a2, ym[1], ym[2], ym[3], ym[4], ym[5], ym[6], ym[7], Am);
        rk4_incr<RM>(a, a2, ym, Am, T(0.5) * h, d);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            d[i] = d1[i] + d[i];
    } else {
        rk4_incr<RM>(a, a2, y, A0, h, df);
        two_halves<RM>(a, a2, y, A0, h, d);
    }
    if constexpr (std::is_same<T, float>::value)
        return err_norm_f(y, d, df, tol);
    else if constexpr (ZONE_NORM && std::is_same<T, double>::value)
        return err_norm_zone(y, d, df, tol);
    else
        return err_norm_d(y, d, df, tol);
}

// Step-size factor after an attempt: 0.9 err^(-1/5) clamped to [0.2, 5]; 5
// for err == 0 and 0.2 for a non-finite err.  FP32 evaluates the power with
// the hardware log2/exp2; FP64 with the correctly rounded pow.
__device__ __forceinline__ float step_factor(float err)
{
    if (!isfinite(err))
        return 0.2f;
    if (err == 0.0f)
        return 5.0f;
    const float f = 0.9f * exp2f(-0.2f * __log2f(err));
    return fminf(5.0f, fmaxf(0.2f, f));
}
__device__ __forceinline__ double step_factor(double err)
{
    if (!isfinite(err))
        return 0.2;
    if (err == 0.0)
        return 5.0;
    const double f = 0.9 * pow(err, -0.2);
    return fmin(5.0, fmax(0.2, f));
}

// The step-size factor of an FP64 zone step of the FP32+Kahan path, taken in
// FP32: it only scales the next trial step, and the FP32 path's accuracy
// target (1e-5) leaves ample room for a factor rounded to FP32.
__device__ __forceinline__ double step_factor_f(double err)
{
    return (double)step_factor((float)err);
}
__device__ __forceinline__ dfloat step_factor_f(dfloat err) { return step_factor(err); }

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

// Event value on a state (y, c): r - target (kind 0), t - (target +
// target_lo) (kind 1; target_lo is the low part of a float-pair end time),
// or z (kind 2, equatorial crossings).
template <bool KAHAN, typename T>
__device__ __forceinline__ T event_value(int kind, T a2, const T y[8], const T c[8], T target,
                                         T target_lo)
{
    if (kind == 0)
        return ks_r(a2, y[1], y[2], y[3]) - target;
    if (kind == 2)
        return KAHAN ? y[3] + c[3] : y[3];
    return KAHAN ? ((y[0] - target) + c[0]) - target_lo : y[0] - target;
}

// Clip an accepted step onto an event surface (Illinois regula falsi on the
// step length eta in (0, h), Phi(eta) = two RK4 half steps from the last
// accepted state (y, c)).  Writes the state on the surface to (ye, ce) and
// returns its step length.  Bracket values s_lo = s(y_old), s_hi = s(y_new).
template <bool KAHAN, typename T, int RM = RHS_INLINE>
__device__ T clip(const T a, const T a2, const T y[8], const T c[8], const T A0[4], const T h,
                  int kind, T target, T target_lo, T s_lo, T s_hi, T stol, T eps, int maxit,
                  T ye[8], T ce[8], uint32_t &nrhs)
{
    T lo = T(0), hi = h;
    T eta_out = h;
    int side = 0;
    T d[8];
    for (int it = 0; it < maxit; ++it) {
        T eta = hi - s_hi * (hi - lo) / (s_hi - s_lo);
        if (!(eta > lo && eta < hi))
            eta = T(0.5) * (lo + hi);
        two_halves<RM>(a, a2, y, A0, eta, d);
        nrhs += 7;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            ye[i] = y[i];
            ce[i] = c[i];
            add_incr<KAHAN>(ye[i], ce[i], d[i]);
        }
        eta_out = eta;
        const T s = event_value<KAHAN>(kind, a2, ye, ce, target, target_lo);
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
    return eta_out;
}

__device__ __forceinline__ float k_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double k_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float k_atan2(dfloat y, dfloat x) { return atan2f(y.hi, x.hi); }
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(double x) { return (float)x; }
__device__ __forceinline__ float to_f(dfloat x) { return x.hi; }

// Clipping tolerances per number type: |s| <= stol * scale, bracket eps * h.
template <typename T> struct Prec;
// ztol: equatorial-crossing root-find (z = 0 has no natural scale of its own).
template <> struct Prec<float> {
    static __device__ __forceinline__ float ztol() { return 6e-8f; }
    static __device__ __forceinline__ float stol() { return 2e-6f; }
    static __device__ __forceinline__ float eps() { return 1e-7f; }
};
template <> struct Prec<double> {
    static __device__ __forceinline__ double ztol() { return 1e-12; }
    static __device__ __forceinline__ double stol() { return 1e-12; }
    static __device__ __forceinline__ double eps() { return 1e-15; }
};
template <> struct Prec<dfloat> {
    static __device__ __forceinline__ dfloat ztol() { return dfloat(1e-12); }
    static __device__ __forceinline__ dfloat stol() { return dfloat(1e-12); }
    static __device__ __forceinline__ dfloat eps() { return dfloat(1e-13); }
};

// Scale of the end-time clipping tolerance.  FP64 and float-float: max(1,
// |t_end|).  FP32 steps: max(1, |t change over the step|) -- the compensated
// time is good to a few units of FP32 roundoff of the step's own increment,
// while a tolerance relative to t_end would leave an end point hundreds of
// time units into an orbit off by a visible fraction of a step.
__device__ __forceinline__ float time_event_scale(float tend, float s_lo, float s_hi)
{
    return fmaxf(1.f, fabsf(s_hi - s_lo));
}
__device__ __forceinline__ double time_event_scale(double tend, double, double)
{
    return fmax(1.0, fabs(tend));
}
__device__ __forceinline__ dfloat time_event_scale(dfloat tend, dfloat, dfloat)
{
    return fmax(dfloat(1.f), fabs(tend));
}

// Conversions used by the FP64 renormalisation.
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(dfloat x) { return (double)x.hi + (double)x.lo; }
template <typename T> __device__ __forceinline__ T from_d(double d) { return (T)d; }
template <> __device__ __forceinline__ dfloat from_d<dfloat>(double d) { return dfloat(d); }

// The rest of an attempt once its error measure err and the increment d of
// the two-half-step solution are known (A0 = accel(y), a2 = a^2): step-size
// control, the compensated update, the termination events, the equatorial
// crossings and the periodic renormalisation.
__device__ __forceinline__ void load_const_full(const TraceParams &P, int64_t id, RayConst &rc);

// LAZY: rc holds the FP32 fields only; the renormalisation loads the FP64
// ones when it runs.
// A step that ended on an event surface whose clipping is left to the clip
// pass: the state stays the one before the step, h its length.
struct ClipRec {
    bool pending = false;
    double s_hi = 0.0;          // event value at the unclipped end of the step
};

//
// ZH (FP64 zone steps of the FP32+Kahan path): the step length lives in FP32
// (*hz; h is its FP64 copy for the arithmetic), and the next one is hz times
// the FP32 factor -- the value that rounding the FP64 product to FP32 gives,
// without the conversions; the tests on err and r compare bit patterns of
// non-negative doubles with integer instructions.  On GB300 each FP64
// compare or conversion occupies the FP64 pipe like an FMA.
template <bool KAHAN, typename T, bool FAST_FACTOR = false, int RM = RHS_INLINE,
          bool LAZY = false, bool ZH = false>
__device__ __forceinline__ int step_post(const RayConst &rc, const TraceParams &P, int64_t id,
                                         const T a, const T a2, const T A0[4], const T d[8],
                                         const T err, T y[8], T c[8], T &h, T &rn,
                                         uint32_t &nrhs, uint32_t &nacc, int &since_renorm,
                                         T *h_taken = nullptr, ClipRec *defer = nullptr,
                                         float *hz = nullptr)
{
    static_assert(!ZH || (FAST_FACTOR && std::is_same<T, double>::value), "FP64 zone steps");
    T fac = T(0);
    float facz = 0.f;
    if constexpr (ZH)
        facz = step_factor((float)err);
    else if constexpr (FAST_FACTOR)
        fac = step_factor_f(err);
    else
        fac = step_factor(err);
    bool accept;
    if constexpr (ZH)
        accept = k_le_nonneg(err, 1.0);
    else
        accept = err <= T(1);
    if (!accept) {
        if constexpr (ZH)
            *hz *= facz;
        else
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
        finite = finite && k_isfinite(yn[i]);
    }
    if (!finite) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            y[i] = yn[i];
            c[i] = cn[i];
        }
        return ST_NONFINITE;
    }
    rn = FAST_FACTOR ? ks_r_zone(a2, yn[1], yn[2], yn[3]) : ks_r(a2, yn[1], yn[2], yn[3]);
    // termination: (yn, cn) becomes the end point of the step, clipped onto
    // the surface when an event fires; h_used is its step length
    const T rcap = RC<T>::rcap(rc);
    const T resc = RC<T>::resc(rc);
    const int maxit = P.clip_maxit;
    // event surfaces to stol x scale; an FP64 (or float-float) zone step of
    // the FP32+Kahan path (FAST_FACTOR), whose end points are good to ~1e-6,
    // places them to 1e-10, which the regula falsi reaches in fewer
    // single-lane iterations than the FP64 path's 1e-12
    const T stol = FAST_FACTOR ? T(1e-10) : Prec<T>::stol();
    // clipping left to the clip pass (not with crossing labels: a crossing in
    // the last step is located on the clipped step)
    const bool defer_ok = defer != nullptr && P.cross == nullptr;
    int st = ST_NONE;
    T h_used = h;
    bool pending = false;
    T s_pend = T(0);
    bool captured, beyond;
    if constexpr (ZH) {
        captured = k_lt_nonneg(rn, rcap);
        beyond = k_gt_nonneg(rn, resc);
    } else {
        captured = rn < rcap;
        beyond = rn > resc;
    }
    if (captured) {
        st = ST_CAPTURED;
        if (defer_ok) {
            pending = true;
            s_pend = rn - rcap;
        } else {
            const T s_lo = event_value<KAHAN>(0, a2, y, c, rcap, T(0));
            h_used = clip<KAHAN, T, RM>(a, a2, y, c, A0, h, 0, rcap, T(0), s_lo, rn - rcap,
                                        stol * rcap, Prec<T>::eps(), maxit, yn, cn, nrhs);
        }
    } else if (beyond && k_fma(yn[1], yn[5], k_fma(yn[2], yn[6], yn[3] * yn[7])) > T(0)) {
        const T s_lo = event_value<KAHAN>(0, a2, y, c, resc, T(0));
        if (s_lo <= T(0)) {
            if (defer_ok) {
                pending = true;
                s_pend = rn - resc;
            } else {
                h_used = clip<KAHAN, T, RM>(a, a2, y, c, A0, h, 0, resc, T(0), s_lo, rn - resc,
                                            stol * resc, Prec<T>::eps(), maxit, yn, cn, nrhs);
            }
        }
        st = ST_ESCAPED;
    } else if (rc.use_t) {
        const T tend = RC<T>::tend(rc), tlo = RC<T>::tendlo(rc);
        const T s_hi = event_value<KAHAN>(1, a2, yn, cn, tend, tlo);
        if ((s_hi > T(0)) != (rc.tpos != 0)) {
            if (defer_ok) {
                pending = true;
                s_pend = s_hi;
            } else {
                const T s_lo = event_value<KAHAN>(1, a2, y, c, tend, tlo);
                const T sc = time_event_scale(tend, s_lo, s_hi);
                h_used = clip<KAHAN, T, RM>(a, a2, y, c, A0, h, 1, tend, tlo, s_lo, s_hi,
                                            stol * sc, Prec<T>::eps(), maxit, yn, cn, nrhs);
            }
            st = ST_ENDTIME;
        }
    }
    if (pending) {
        defer->pending = true;
        defer->s_hi = to_d(s_pend);
        return st;
    }
    // equatorial crossings within [y, end point]
    if (P.cross) {
        const T z0 = y[3], z1 = yn[3];
        if ((z0 > T(0) && !(z1 > T(0))) || (z0 < T(0) && !(z1 < T(0)))) {
            const int64_t n = P.n;
            const int slot = isnan(P.cross[id]) ? 0 : (isnan(P.cross[2 * n + id]) ? 1 : 2);
            if (slot < 2) {
                T yc[8], cc[8];
                // scale of z at the crossing: the nearer end of the step
                const T r0 = ks_r(a2, y[1], y[2], y[3]);
                const T r1 = ks_r(a2, yn[1], yn[2], yn[3]);
                clip<KAHAN, T, RM>(a, a2, y, c, A0, h_used, 2, T(0), T(0), z0, z1,
                            Prec<T>::ztol() * (T(1) + fmin(r0, r1)), Prec<T>::eps(), maxit, yc,
                            cc, nrhs);
                const T rcx = ks_r(a2, yc[1], yc[2], yc[3]);
                float ph = k_atan2(yc[2], yc[1]) - k_atan2(a, rcx);
                if (ph <= -3.14159265f)
                    ph += 6.28318531f;
                else if (ph > 3.14159265f)
                    ph -= 6.28318531f;
                P.cross[(2 * slot) * n + id] = to_f(rcx);
                P.cross[(2 * slot + 1) * n + id] = ph;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        y[i] = yn[i];
        c[i] = cn[i];
    }
    if (h_taken)
        *h_taken = h_used;
    if (st != ST_NONE)
        return st;
    if (P.renorm_every > 0 && ++since_renorm >= P.renorm_every) {
        since_renorm = 0;
        double k[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            k[j] = to_d(y[4 + j]) + (KAHAN ? to_d(c[4 + j]) : 0.0);
        RayConst rf = rc;
        if (LAZY)
            load_const_full(P, id, rf);
        const KSPoint p = ks_point(rf.a, to_d(y[1]) + (KAHAN ? to_d(c[1]) : 0.0),
                                   to_d(y[2]) + (KAHAN ? to_d(c[2]) : 0.0),
                                   to_d(y[3]) + (KAHAN ? to_d(c[3]) : 0.0));
        if (solve_kt(p, k, rf.u2_0, 0)) {
            y[4] = from_d<T>(k[0]);
            c[4] = KAHAN ? from_d<T>(k[0] - to_d(y[4])) : T(0);
        }
    }
    if constexpr (ZH)
        *hz *= facz;
    else
        h *= fac;
    return ST_NONE;
}

// One attempted step with events.  (y, c) is the lane state; h the trial
// step; rn receives r of the new state when a step is accepted.  Returns a
// status code when the geodesic terminates, ST_NONE otherwise.
template <bool KAHAN, typename T, bool FAST_FACTOR = false, int RM = RHS_INLINE>
__device__ __forceinline__ int step_once(const RayConst &rc, const TraceParams &P, int64_t id,
                                         const T tol, T y[8], T c[8], T &h, T &rn,
                                         uint32_t &nrhs, uint32_t &nacc, int &since_renorm,
                                         T *h_taken = nullptr, ClipRec *defer = nullptr)
{
    const T a = RC<T>::a(rc);
    const T a2 = a * a;
    T A0[4];
    rhs<RM>(a, a2, y[1], y[2], y[3], y[4], y[5], y[6], y[7], A0);
    T d[8];
    // FP64 zone steps of the FP32+Kahan path (FAST_FACTOR): the cheaper measure
    const T err = attempt<RM, FAST_FACTOR>(a, a2, y, A0, h, tol, d);
    nrhs += 11;
    return step_post<KAHAN, T, FAST_FACTOR, RM>(rc, P, id, a, a2, A0, d, err, y, c, h, rn, nrhs,
                                                nacc, since_renorm, h_taken, defer);
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
    KSPoint kp;                 // the metric's pieces at the start point
    bool have_kp = false;
    if (P.mode == MODE_CAMERA || P.mode == MODE_POINTS) {
        double al, be, r_obs, si, ci;
        if (P.mode == MODE_CAMERA) {
            const int64_t pix = P.index ? P.index[id] : id;
            int lo = 0, hi = P.ncam - 1;
            while (lo < hi) {   // last camera with offset <= pix
                const int mid = (lo + hi + 1) >> 1;
                if (P.cams[mid].offset <= pix)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const CamDev cam = P.cams[lo];
            a = cam.a;
            const int64_t local = pix - cam.offset;
            const int64_t p = local % cam.nx, q = local / cam.nx;
            // pixel centre -w + (p + 1/2) 2w / nx = (2p + 1 - nx) (w / nx), the
            // first factor an exact integer (one refined reciprocal, no
            // division: on GB300 an IEEE FP64 division costs a dozen FP64
            // instructions)
            al = (double)(2 * p + 1 - cam.nx) * (cam.w * k_rcp((double)cam.nx));
            be = (double)(2 * q + 1 - cam.ny) * (cam.w * k_rcp((double)cam.ny));
            si = cam.sin_incl;
            ci = cam.cos_incl;
            r_obs = cam.r_obs;
        } else {
            al = P.points[4 * id];
            be = P.points[4 * id + 1];
            a = P.points[4 * id + 2];
            sincos(P.points[4 * id + 3], &si, &ci);
            r_obs = P.r_obs;
        }
        y[0] = 0.0;
        y[1] = r_obs * si - be * ci;
        y[2] = al;
        y[3] = r_obs * ci + be * si;
        y[5] = -si;
        y[6] = 0.0;
        y[7] = -ci;
        y[4] = 0.0;
        kp = ks_point(a, y[1], y[2], y[3]);
        have_kp = true;
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
            kp = ks_point(a, y[1], y[2], y[3]);
            have_kp = true;
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
    const double rh = 1.0 + k_sqrt(fmax(0.0, 1.0 - a * a));
    rc.rcap = 1.01 * rh;
    rc.zone_r = P.fp64_zone * rh;
    const double tend = P.t_end_each ? P.t_end_each[id] : P.t_end;
    rc.use_t = isfinite(tend) ? 1 : 0;
    rc.tend = tend;
    rc.tpos = (y[0] - tend) > 0.0 ? 1 : 0;
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        finite = finite && k_isfinite(y[i]);
    if (st == ST_NONE && !finite)
        st = ST_NONFINITE;
    // r, f and l at the start point (the camera branch has them already)
    if (finite && !have_kp)
        kp = ks_point(a, y[1], y[2], y[3]);
    // (kp.r = r^2 rsqrt(r^2) is NaN where r^2 is 0 or inf; ks_r gives 0 / NaN there)
    const double r0 = !finite ? 0.0 : (k_isfinite(kp.r) ? kp.r : ks_r(a * a, y[1], y[2], y[3]));
    rc.resc = P.r_escape > 0.0 ? P.r_escape : (P.r_escape == 0.0 ? r0 : INFINITY);
    rc.xi = 0.0;
    if (st == ST_NONE) {
        rc.u2_0 = norm2(kp, y + 4);
        // E = -p_t and L_z = x p_y - y p_x with p = eta k + f l (l.k)
        const double L = y[4] + kp.lx * y[5] + kp.ly * y[6] + kp.lz * y[7];
        const double E = y[4] - kp.f * L;
        const double Lz = y[1] * (y[6] + kp.f * kp.ly * L) - y[2] * (y[5] + kp.f * kp.lx * L);
        rc.xi = Lz * k_rcp(E);
        if (r0 < rc.rcap)
            st = ST_CAPTURED;
    }
    finish_const(rc);
    return st;
}

// Prograde ISCO radius (Bardeen, Press & Teukolsky 1972).
__device__ __forceinline__ double r_isco(double a)
{
    const double z1 = 1.0 + cbrt(1.0 - a * a) * (cbrt(1.0 + a) + cbrt(1.0 - a));
    const double z2 = sqrt(3.0 * a * a + z1 * z1);
    return 3.0 + z2 - sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
}

// Redshift of a prograde Keplerian emitter at radius r seen along a ray with
// xi = L_z / E: g = 1 / (u^t (1 - Omega xi)), Omega = 1/(r^{3/2} + a),
// u^t = (r^{3/2} + a) / (r^{3/4} sqrt(r^{3/2} - 3 r^{1/2} + 2a)); NaN inside
// the ISCO or for a missing crossing.
__device__ __forceinline__ float redshift_label(double a, double r, double xi)
{
    if (!(r >= r_isco(a)))
        return __int_as_float(0x7fc00000);
    const double s = sqrt(r), r32 = r * s;
    const double ut = (r32 + a) / (sqrt(s) * s * sqrt(r32 - 3.0 * s + 2.0 * a));
    const double Om = 1.0 / (r32 + a);
    return (float)(1.0 / (ut * (1.0 - Om * xi)));
}

__device__ __forceinline__ void clear_cross(const TraceParams &P, int64_t id)
{
    if (P.cross) {
#pragma unroll
        for (int j = 0; j < 5; ++j)
            P.cross[j * P.n + id] = __int_as_float(0x7fc00000);
    }
}

__device__ __forceinline__ void write_out(const TraceParams &P, int64_t id, const double y[8],
                                          int st, uint32_t nsteps, double a, double xi)
{
    if (P.cross)
        P.cross[4 * P.n + id] = redshift_label(a, (double)P.cross[id], xi);
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

// A stop request: the launch's wall-time budget ran out, or the host set the
// context's abort flag (mapped pinned memory, read at system scope so that a
// host write made while the kernel runs becomes visible).
__device__ __forceinline__ bool stop_requested(const TraceParams &P, unsigned long long t_start)
{
    if (P.budget_ns && (global_ns() - t_start) > P.budget_ns)
        return true;
    if (P.abort) {
        int32_t v;
        asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(P.abort) : "memory");
        return v != 0;
    }
    return false;
}

// Zone steps of an FP32+Kahan geodesic (inside the zone r < fp64_zone r_h,
// where f l l is large) run out of line, so that their registers do not raise
// the register count of the loop around them; the lane state travels by
// value so that the caller's arrays stay in registers.
struct LaneF {
    float y[8], c[8];
    float h, rnow;
};
struct ZoneResult {
    LaneF s;
    int st;
    uint32_t nrhs, nacc;
    int since_renorm;
    ClipRec clip;               // the step's clipping was deferred (state before it)
};

// FP64 state held in the (y, c) registers of a lane as bit patterns (low
// word in y, high word in c): consecutive zone steps of one geodesic keep
// its FP64 state instead of rounding it to an FP32 pair after every attempt
// (on GB300 each conversion costs the FP64 pipe as much as an FMA).
__device__ __forceinline__ double d_from_bits(float lo, float hi)
{
    return __hiloint2double(__float_as_int(hi), __float_as_int(lo));
}
__device__ __forceinline__ void d_to_bits(double v, float &lo, float &hi)
{
    lo = __int_as_float(__double2loint(v));
    hi = __int_as_float(__double2hiint(v));
}

struct Y8d {
    double v[8];
};
struct ZoneResultD {
    Y8d y;
    float h, rnow;
    int st;
    uint32_t nrhs, nacc;
    int since_renorm;
    ClipRec clip;               // the step's clipping was deferred (state before it)
};

// One FP64 zone attempt on an FP64 state (zone phase); the lane keeps the
// state in FP64 between attempts.
template <int RM>
static __device__ __noinline__ ZoneResultD zone_step_d(const RayConst rc, const TraceParams &P,
                                                      int64_t id, Y8d s, float h, float rnow,
                                                      int since_renorm)
{
    double cd[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        cd[i] = 0.0;
    const double a = rc.a;
    const double a2 = a * a;
    // the step length stays FP32 (hz); r is written by an accepted step only
    const double hd = (double)h;
    float hz = h;
    double rd = -1.0;
    double A0[4];
    rhs<RM>(a, a2, s.v[1], s.v[2], s.v[3], s.v[4], s.v[5], s.v[6], s.v[7], A0);
    double d[8];
    const double err = attempt<RM, true>(a, a2, s.v, A0, hd, P.tol, d);
    ZoneResultD R;
    R.nrhs = 11;
    R.nacc = 0;
    double hu = hd;
    R.st = step_post<false, double, true, RM, false, true>(
        rc, P, id, a, a2, A0, d, err, s.v, cd, hu, rd, R.nrhs, R.nacc, since_renorm, nullptr,
        P.clipq ? &R.clip : nullptr, &hz);
    R.y = s;
    R.h = hz;
    R.rnow = __double2hiint(rd) >= 0 ? (float)rd : rnow;
    R.since_renorm = since_renorm;
    return R;
}

// One FP64 zone attempt taken by two lanes of a warp (zone phase, its tail):
// the owner holds the geodesic; its helper, an idle lane, receives the state,
// the trial step and the spin, and computes the full step of h while the
// owner computes the first half step (the same instructions on other data,
// so the warp pays for one); the owner then takes the second half step and
// reads the full step's increment back.  On GB300 an FP64 warp instruction
// costs the same whatever its active lanes, so an attempt's latency falls
// from eleven right-hand sides to eight.  The operations are those of
// step_once (right-hand sides, RK4 steps, error measure, step_post), so the
// result is the owner's zone_step_d result bit for bit.  `tmask` holds the
// owners and their helpers; partner is the other lane of the pair.  A
// helper's result is meaningless.
template <int RM>
static __device__ __noinline__ ZoneResultD zone_step_team(const RayConst rc, const TraceParams &P,
                                                         int64_t id, Y8d s, float h, float rnow,
                                                         int since_renorm, bool helper,
                                                         int partner, unsigned tmask)
{
    const int lane = threadIdx.x & 31;
    const int src = helper ? partner : lane;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        s.v[i] = __shfl_sync(tmask, s.v[i], src);
    const float hs = __shfl_sync(tmask, h, src);
    const double a = __shfl_sync(tmask, rc.a, src);
    const double a2 = a * a;
    const double hd = (double)hs;
    float hz = hs;
    double rd = -1.0;
    double A0[4];
    rhs<RM>(a, a2, s.v[1], s.v[2], s.v[3], s.v[4], s.v[5], s.v[6], s.v[7], A0);
    // helper: the full step of h; owner: the first half step
    double dp[8];
    rk4_incr<RM>(a, a2, s.v, A0, helper ? hd : 0.5 * hd, dp);
    double d[8];
    if (!helper) {
        double ym[8], Am[4], d2[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            ym[i] = s.v[i] + dp[i];
        rhs<RM>(a, a2, ym[1], ym[2], ym[3], ym[4], ym[5], ym[6], ym[7], Am);
        rk4_incr<RM>(a, a2, ym, Am, 0.5 * hd, d2);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            d[i] = dp[i] + d2[i];
    }
    double df[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        df[i] = __shfl_sync(tmask, dp[i], helper ? lane : partner);
    ZoneResultD R;
    R.nrhs = 0;
    R.nacc = 0;
    R.st = ST_NONE;
    if (!helper) {
        const double err = err_norm_zone(s.v, d, df, P.tol);
        R.nrhs = 11;
        double cd[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            cd[i] = 0.0;
        double hu = hd;
        R.st = step_post<false, double, true, RM, false, true>(
            rc, P, id, a, a2, A0, d, err, s.v, cd, hu, rd, R.nrhs, R.nacc, since_renorm, nullptr,
            P.clipq ? &R.clip : nullptr, &hz);
    }
    R.y = s;
    R.h = hz;
    R.rnow = __double2hiint(rd) >= 0 ? (float)rd : rnow;
    R.since_renorm = since_renorm;
    return R;
}

// One zone attempt in float-float arithmetic (zone_prec KERR_ZONE_F32X2):
// the compensated pair (y, c) is already a float-float number, so no FP64
// instruction is needed.
template <int RM>
static __device__ __noinline__ ZoneResult zone_step_df(const RayConst rc, const TraceParams &P,
                                                       int64_t id, LaneF s, int since_renorm)
{
    dfloat yd[8], cd[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        yd[i] = quick_two_sum(s.y[i], s.c[i]);
        cd[i] = dfloat(0.f, 0.f);
    }
    dfloat hd(s.h, 0.f), rd(s.rnow, 0.f);
    ZoneResult R;
    R.nrhs = 0;
    R.nacc = 0;
    R.st = step_once<false, dfloat, true, RM>(rc, P, id, dfloat((float)P.tol), yd, cd, hd, rd,
                                              R.nrhs, R.nacc, since_renorm, nullptr,
                                              P.clipq ? &R.clip : nullptr);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        R.s.y[i] = yd[i].hi;
        R.s.c[i] = yd[i].lo;
    }
    R.s.h = hd.hi;
    R.s.rnow = rd.hi;
    R.since_renorm = since_renorm;
    return R;
}

// Spin of geodesic id: its camera's (camera mode) or the context's.
__device__ __forceinline__ double geodesic_spin(const TraceParams &P, int64_t id)
{
    if (P.mode == MODE_POINTS)
        return P.points[4 * id + 2];
    if (P.mode != MODE_CAMERA)
        return P.a;
    const int64_t pix = P.index ? P.index[id] : id;
    int lo = 0, hi = P.ncam - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.cams[mid].offset <= pix)
            lo = mid;
        else
            hi = mid - 1;
    }
    return P.cams[lo].a;
}

// Statistics: warp reduction, one atomic per counter per warp.
struct Counters {
    uint32_t geo = 0, att = 0, acc = 0, rhs32 = 0, rhs64 = 0, att64 = 0, def = 0, req = 0;
    uint32_t st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t r32z = 0, a32z = 0, clips = 0, clip_rhs = 0;
    __device__ __forceinline__ void status(int s)
    {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            st[j] += (s == j) ? 1u : 0u;
    }
    __device__ __forceinline__ void flush(unsigned long long *stats) const
    {
        const unsigned FULL = 0xffffffffu;
        auto wsum = [&](uint32_t v) -> unsigned long long {
            unsigned long long x = v;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                x += __shfl_xor_sync(FULL, x, o);
            return x;
        };
        const unsigned long long v[8] = {wsum(geo),   wsum(att),   wsum(acc), wsum(rhs32),
                                         wsum(rhs64), wsum(att64), wsum(def), wsum(req)};
        unsigned long long w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            w[j] = wsum(st[j]);
        const unsigned long long u[4] = {wsum(r32z), wsum(a32z), wsum(clips), wsum(clip_rhs)};
        if ((threadIdx.x & 31) == 0) {
            const int slot[8] = {SC_GEODESICS, SC_ATTEMPTS, SC_ACCEPTED, SC_RHS32,
                                 SC_RHS64,     SC_ATT64,    SC_DEFERRED, SC_REQUEUED};
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (v[j])
                    atomicAdd(stats + slot[j], v[j]);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (w[j])
                    atomicAdd(stats + SC_STATUS + j, w[j]);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (u[j])
                    atomicAdd(stats + SC_RHS32_ZONE + j, u[j]);
        }
    }
};

// The lowest k set bits of m (k <= popc(m)).
__device__ __forceinline__ unsigned low_bits(unsigned m, int k)
{
    unsigned r = 0;
    for (int j = 0; j < k && m; ++j) {
        const unsigned b = m & (0u - m);
        r |= b;
        m ^= b;
    }
    return r;
}
// Index of the k-th (0-based) set bit of m (k < popc(m)).
__device__ __forceinline__ int nth_bit(unsigned m, int k)
{
    for (int j = 0; j < k; ++j)
        m &= m - 1u;
    return __ffs(m) - 1;
}

// Warp-aggregated claim of `cnt` consecutive items from a counter; every
// lane of the warp gets the base.
__device__ __forceinline__ unsigned long long warp_claim(unsigned long long *ctr, unsigned mask)
{
    const unsigned FULL = 0xffffffffu;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if ((int)(threadIdx.x & 31) == leader)
        base = atomicAdd(ctr, (unsigned long long)__popc(mask));
    return __shfl_sync(FULL, base, leader);
}

// ---------------------------------------------------------------------------
// Zone-phase queue.  The deferred geodesics sit in a ring of zcap entries:
// index i lives in slot i mod zcap.  The FP32 phase writes indices
// 0 .. n0 - 1 (n0 = min(zcount, zcap)); the zone phase re-queues at
// n0 + zpush (zpush counts re-queued geodesics) and claims at zhead.  A
// writer fills the entry and then publishes seq = i + 1 (release); a reader waits for that value (acquire), reads, and
// sets seq = 0, which a writer of the slot's next index waits for.  The ring
// never holds more geodesics than the phase started with (each is either
// in a lane or in the ring), so zcap >= that count keeps indices i and
// i + zcap from meeting.  Both waits are bounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Waits (bounded: about 2^22 polls, ~0.5 s) until *p == want.
__device__ __forceinline__ bool wait_seq(const uint32_t *p, uint32_t want)
{
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        if (ld_acquire(p) == want)
            return true;
        __nanosleep(64);
    }
    return false;
}

// Warp-aggregated claim of up to popc(mask) indices below the queue tail
// t0 + *pushed.  Returns the first index; *take (warp-uniform) is how many
// were claimed and *empty whether the leader saw head >= tail.
__device__ __forceinline__ unsigned long long warp_claim_queue(unsigned long long *head,
                                                               unsigned long long t0,
                                                               const unsigned long long *pushed,
                                                               unsigned mask, unsigned *take,
                                                               bool *empty)
{
    const unsigned FULL = 0xffffffffu;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    unsigned got = 0;
    int emp = 0;
    if ((int)(threadIdx.x & 31) == leader) {
        unsigned long long h = ld_relaxed(head);
        for (int tries = 0; tries < 64; ++tries) {
            const unsigned long long t = t0 + (pushed ? ld_relaxed(pushed) : 0ull);
            if (h >= t) {
                emp = 1;
                break;
            }
            const unsigned long long k =
                min((unsigned long long)__popc(mask), t - h);
            const unsigned long long old = atomicCAS(head, h, h + k);
            if (old == h) {
                base = h;
                got = (unsigned)k;
                break;
            }
            h = old;
        }
    }
    base = __shfl_sync(FULL, base, leader);
    *take = __shfl_sync(FULL, got, leader);
    *empty = __shfl_sync(FULL, emp, leader) != 0;
    return base;
}

// ===========================================================================
// FP64 path: one persistent kernel, set-up and output inline.
// ===========================================================================
template <int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) trace_f64_kernel(const TraceParams P)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned long long n_items = (unsigned long long)P.n;
    if (P.n_dev && *P.n_dev < n_items)
        n_items = *P.n_dev;
    bool has = false, drained = false, timed_out = false;
    int64_t id = 0;
    RayConst rc;
    double y[8], c[8];
    double h = 0.0, rnow = 0.0;
    uint32_t nsteps = 0;
    int since_renorm = 0;
    Counters C;
    const unsigned long long t_start = global_ns();
    uint32_t iter = 0;
    // stored solution (dense output): affine parameter and state after every
    // accepted step, up to traj_cap records per geodesic
    double lam = 0.0;
    int32_t ntraj = 0;
    auto record = [&](double l, const double s[8]) {
        if (P.traj && ntraj < P.traj_cap) {
            double *dst = P.traj + ((size_t)id * P.traj_cap + ntraj) * 9;
            dst[0] = l;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                dst[1 + i] = s[i];
            ++ntraj;
            P.traj_count[id] = ntraj;
        }
    };
    for (;;) {
        const unsigned need = __ballot_sync(FULL, !has);
        if (need && !drained) {
            const unsigned long long base = warp_claim(P.head, need);
            if (base + __popc(need) >= n_items)
                drained = true;
            if (!has) {
                const unsigned long long my = base + __popc(need & lt_mask);
                if (my < n_items) {
                    id = (int64_t)my;
                    if (P.traj)
                        P.traj_count[id] = 0;
                    const int st0 = init_geodesic(P, id, y, rc);
                    clear_cross(P, id);
                    ++C.geo;
                    if (st0 != ST_NONE || timed_out) {
                        const int st = st0 != ST_NONE ? st0 : ST_TIMEOUT;
                        write_out(P, id, y, st, 0, rc.a, rc.xi);
                        C.status(st);
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            c[i] = 0.0;
                        h = P.h0;
                        nsteps = 0;
                        since_renorm = 0;
                        lam = 0.0;
                        ntraj = 0;
                        record(lam, y);
                        has = true;
                    }
                }
            }
        }
        if (!__any_sync(FULL, has)) {
            if (drained)
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
                ++C.att;
                ++C.att64;
                uint32_t r = 0;
                double taken = 0.0;
                // right-hand sides out of line: one copy keeps the kernel in
                // the instruction cache (same arithmetic as inline)
                st = step_once<false, double, false, RHS_CALL>(rc, P, id, P.tol, y, c, h, rnow,
                                                               r, C.acc, since_renorm, &taken);
                C.rhs64 += r;
                if (taken != 0.0) {
                    lam += taken;
                    record(lam, y);
                }
            }
            if (st != ST_NONE) {
                write_out(P, id, y, st, nsteps, rc.a, rc.xi);
                C.status(st);
                has = false;
            }
        }
        if ((P.budget_ns || P.abort) && ((++iter & 31u) == 0) && !timed_out) {
            bool over = false;
            if (lane == 0)
                over = stop_requested(P, t_start);
            timed_out = __shfl_sync(FULL, over, 0);
        }
    }
    C.flush(P.stats);
}

// ===========================================================================
// FP32+Kahan path: three launches.
//   f32_setup_kernel   FP64 initial states (whole warps, coalesced) split
//                      into FP32 pairs + per-geodesic constants in scratch;
//                      geodesics that end at once get their status here.
//   trace_f32_kernel   PHASE 0: persistent FP32 stepping, no FP64 arithmetic
//                      (geodesics entering the zone are deferred; the zone
//                      buffer holds one entry per geodesic);
//                      PHASE 1: continues the deferred zone geodesics.
//   f32_finish_kernel  folds the compensated pairs into FP64 outputs and
//                      computes the FP64 diagnostics (whole warps).
// ===========================================================================
// Appends the geodesics of the warp whose clipping was deferred to the clip
// queue (warp-aggregated; every lane of the warp calls this): FP32 clips from
// the front, zone-arithmetic clips from the back.  Each geodesic ends once,
// so the two ends never meet.
// Clip-queue entries of zone clips whose stored state is FP64 bit patterns
// (zone phase) rather than an FP32 pair carry this bit.
constexpr int64_t kClipFP64State = 1ll << 62;

__device__ __forceinline__ void enqueue_clips(const TraceParams &P, bool pend32, bool pend64,
                                              int64_t id, bool fp64_state = false)
{
    const unsigned FULL = 0xffffffffu;
    const unsigned lt_mask = (1u << (threadIdx.x & 31)) - 1u;
    const unsigned m32 = __ballot_sync(FULL, pend32);
    if (m32) {
        const unsigned long long b = warp_claim(P.cq32, m32);
        if (pend32)
            P.clipq[b + __popc(m32 & lt_mask)] = id;
    }
    const unsigned m64 = __ballot_sync(FULL, pend64);
    if (m64) {
        const unsigned long long b = warp_claim(P.cq64, m64);
        if (pend64)
            P.clipq[P.n - 1 - (int64_t)(b + __popc(m64 & lt_mask))] =
                fp64_state ? (id | kClipFP64State) : id;
    }
}

// Number of geodesics of a launch: n, or the device-side count when given.
__device__ __forceinline__ int64_t live_count(const TraceParams &P)
{
    if (P.n_dev && (int64_t)*P.n_dev < P.n)
        return (int64_t)*P.n_dev;
    return P.n;
}

static __global__ void __launch_bounds__(256) f32_setup_kernel(const TraceParams P)
{
    const int64_t n = P.n;
    const int64_t live = live_count(P);
    Counters C;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < live;
         id += (int64_t)gridDim.x * blockDim.x) {
        double yd[8];
        RayConst rc;
        const int st0 = init_geodesic(P, id, yd, rc);
        ++C.geo;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float hi = (float)yd[i];
            P.s_state[i * n + id] = hi;
            P.s_state[(8 + i) * n + id] = k_isfinite(yd[i]) ? (float)(yd[i] - (double)hi) : 0.0f;
        }
        P.s_const[KC_A * n + id] = rc.af;
        P.s_const[KC_RCAP * n + id] = rc.rcapf;
        P.s_const[KC_RESC * n + id] = rc.rescf;
        P.s_const[KC_ZONE * n + id] = rc.zonef;
        P.s_const[KC_TEND * n + id] = rc.tendf;
        P.s_const[KC_TENDLO * n + id] = rc.tendlo;
        P.s_const[KC_U2 * n + id] = (float)rc.u2_0;
        P.s_const[KC_FLAGS * n + id] = __int_as_float((rc.use_t ? 1 : 0) | (rc.tpos ? 2 : 0));
        P.s_const[KC_XI * n + id] = (float)rc.xi;
        clear_cross(P, id);
        P.status[id] = st0;
        P.steps[id] = 0;
        if (st0 != ST_NONE)
            C.status(st0);
    }
    // every lane of every warp reaches here (grid-stride loop above)
    C.flush(P.stats);
}

static __global__ void __launch_bounds__(256) f32_finish_kernel(const TraceParams P)
{
    const int64_t n = P.n;
    const int64_t live = live_count(P);
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < live;
         id += (int64_t)gridDim.x * blockDim.x) {
        double y[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            y[i] = (double)P.s_state[i * n + id] + (double)P.s_state[(8 + i) * n + id];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            P.x_out[j * n + id] = y[j];
            P.k_out[j * n + id] = y[4 + j];
        }
        if (P.cross)
            P.cross[4 * n + id] = redshift_label(geodesic_spin(P, id), (double)P.cross[id],
                                                 (double)P.s_const[KC_XI * n + id]);
        if (P.diag) {
            const int st = P.status[id];
            float cst[4];
            if (st == ST_INVALID_IC || st == ST_NONFINITE) {
                cst[0] = cst[1] = cst[2] = cst[3] = __int_as_float(0x7fc00000);
            } else {
                constants(geodesic_spin(P, id), y, cst);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                P.diag[j * n + id] = cst[j];
        }
    }
}

// Event surface of a geodesic that ended with status st: kind (0: r, 1: t),
// target value, its low part (float-pair end time) and the scale of the
// clipping tolerance -- as chosen by step_post.
template <typename T>
__device__ __forceinline__ void event_of(const RayConst &rc, int st, int &kind, T &target, T &tlo,
                                         T &scale)
{
    tlo = T(0);
    if (st == ST_CAPTURED) {
        kind = 0;
        target = RC<T>::rcap(rc);
        scale = target;
    } else if (st == ST_ESCAPED) {
        kind = 0;
        target = RC<T>::resc(rc);
        scale = target;
    } else {
        kind = 1;
        target = RC<T>::tend(rc);
        tlo = RC<T>::tendlo(rc);
        scale = fmax(T(1), fabs(target));
    }
}

__device__ __forceinline__ void load_const_f32(const TraceParams &P, int64_t id, RayConst &rc);

// The deferred clip of a geodesic whose last step was an FP32 step: the same
// Illinois iteration step_post runs in place (FP32, compensated state).
__device__ __forceinline__ void clip_end_f32(const TraceParams &P, int64_t id, int st, float y[8],
                                             float c[8], uint32_t &nrhs)
{
    RayConst rc;
    load_const_f32(P, id, rc);
    const float a = rc.af, a2 = a * a;
    float A0[4];
    rhs<RHS_CALL>(a, a2, y[1], y[2], y[3], y[4], y[5], y[6], y[7], A0);
    ++nrhs;
    int kind = 0;
    float target, tlo, scale;
    event_of<float>(rc, st, kind, target, tlo, scale);
    const float s_lo = event_value<true>(kind, a2, y, c, target, tlo);
    const float s_hi = (float)P.clip_shi[id];
    if (kind == 1)
        scale = time_event_scale(target, s_lo, s_hi);
    float ye[8], ce[8];
    clip<true, float, RHS_CALL>(a, a2, y, c, A0, P.clip_h[id], kind, target, tlo, s_lo, s_hi,
                                Prec<float>::stol() * scale, Prec<float>::eps(), P.clip_maxit,
                                ye, ce, nrhs);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        y[i] = ye[i];
        c[i] = ce[i];
    }
}

__device__ __forceinline__ double zfold(float y, float c, double) { return (double)y + (double)c; }
__device__ __forceinline__ dfloat zfold(float y, float c, dfloat) { return quick_two_sum(y, c); }
__device__ __forceinline__ void zsplit(double v, float &y, float &c)
{
    y = (float)v;
    c = (float)(v - (double)y);
}
__device__ __forceinline__ void zsplit(dfloat v, float &y, float &c)
{
    y = v.hi;
    c = v.lo;
}

// The deferred clip of a geodesic whose last step was a zone step (FP64 or
// float-float): the zone step's arithmetic and its 1e-10 tolerance.
template <typename T>
__device__ void clip_end_zone(const TraceParams &P, int64_t id, int st, float y[8], float c[8],
                              bool fp64_state, uint32_t &nrhs)
{
    RayConst rc;
    load_const_full(P, id, rc);
    T yd[8], cd[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if constexpr (std::is_same<T, double>::value)
            yd[i] = fp64_state ? d_from_bits(y[i], c[i]) : zfold(y[i], c[i], T(0));
        else
            yd[i] = zfold(y[i], c[i], T(0));
        cd[i] = T(0);
    }
    const T a = RC<T>::a(rc), a2 = a * a;
    T A0[4];
    rhs<RHS_CALL>(a, a2, yd[1], yd[2], yd[3], yd[4], yd[5], yd[6], yd[7], A0);
    ++nrhs;
    int kind = 0;
    T target, tlo, scale;
    event_of<T>(rc, st, kind, target, tlo, scale);
    const T s_lo = event_value<false>(kind, a2, yd, cd, target, tlo);
    T ye[8], ce[8];
    clip<false, T, RHS_CALL>(a, a2, yd, cd, A0, T(P.clip_h[id]), kind, target, tlo, s_lo,
                             from_d<T>(P.clip_shi[id]), T(1e-10) * scale, Prec<T>::eps(),
                             P.clip_maxit, ye, ce, nrhs);
#pragma unroll
    for (int i = 0; i < 8; ++i)
        zsplit(ye[i], y[i], c[i]);
}

// Clip pass of the FP32 path: finishes, with whole warps, the geodesics whose
// last step crossed an event surface -- work that ran for one lane at a time
// while the rest of its warp waited when it was done inside the stepping
// loops.  Threads below the FP32 count take FP32 clips, the others zone
// clips, so a warp mixes the two at most once.
static __global__ void __launch_bounds__(128) f32_clip_kernel(const TraceParams P)
{
    const int64_t n = P.n;
    const unsigned long long n32 = *P.cq32, n64 = *P.cq64;
    const unsigned long long total = n32 + n64;
    Counters C;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         k < total; k += (unsigned long long)gridDim.x * blockDim.x) {
        const bool fp32 = k < n32;
        const int64_t q = fp32 ? P.clipq[k] : P.clipq[n - 1 - (int64_t)(k - n32)];
        const bool fp64_state = (q & kClipFP64State) != 0;
        const int64_t id = q & ~kClipFP64State;
        const int st = P.status[id];
        float y[8], c[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            y[i] = P.s_state[i * n + id];
            c[i] = P.s_state[(8 + i) * n + id];
        }
        uint32_t nrhs = 0;
        if (fp32)
            clip_end_f32(P, id, st, y, c, nrhs);
        else if (P.zone_df)
            clip_end_zone<dfloat>(P, id, st, y, c, false, nrhs);
        else
            clip_end_zone<double>(P, id, st, y, c, fp64_state, nrhs);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            P.s_state[i * n + id] = y[i];
            P.s_state[(8 + i) * n + id] = c[i];
        }
        ++C.clips;
        C.clip_rhs += nrhs;
    }
    // every thread of the grid reaches here (grid-stride loop above)
    C.flush(P.stats);
}

// FP32 lane constants from the planes (PHASE 0) -- no FP64 arithmetic.
__device__ __forceinline__ void load_const_f32(const TraceParams &P, int64_t id, RayConst &rc)
{
    const int64_t n = P.n;
    rc.af = P.s_const[KC_A * n + id];
    rc.rcapf = P.s_const[KC_RCAP * n + id];
    rc.rescf = P.s_const[KC_RESC * n + id];
    rc.zonef = P.s_const[KC_ZONE * n + id];
    rc.tendf = P.s_const[KC_TEND * n + id];
    rc.tendlo = P.s_const[KC_TENDLO * n + id];
    const int fl = __float_as_int(P.s_const[KC_FLAGS * n + id]);
    rc.use_t = fl & 1;
    rc.tpos = (fl >> 1) & 1;
}

// Full constants (FP64 fields too) for the zone phase and the clip pass.
__device__ __forceinline__ void load_const_full(const TraceParams &P, int64_t id, RayConst &rc)
{
    const int64_t n = P.n;
    load_const_f32(P, id, rc);
    rc.a = geodesic_spin(P, id);
    const double rh = 1.0 + sqrt(fmax(0.0, 1.0 - rc.a * rc.a));
    rc.rcap = 1.01 * rh;
    rc.zone_r = P.fp64_zone * rh;
    rc.resc = (double)rc.rescf;
    rc.tend = P.t_end_each ? P.t_end_each[id] : P.t_end;
    rc.u2_0 = (double)P.s_const[KC_U2 * n + id];
    rc.alo = (float)(rc.a - (double)rc.af);            // low parts for float-float steps
    rc.rcaplo = (float)(rc.rcap - (double)rc.rcapf);
}

// TEAM (FP64 zone phase): once at most half as many geodesics remain as the
// grid has lanes, every warp keeps at most 16 of them (the rest go back to
// the queue) and pairs each with an idle lane for its zone attempts
// (zone_step_team).
template <int PHASE, int BLOCK, int MINB, int RM = RHS_INLINE, bool TEAM = false>
__global__ void __launch_bounds__(BLOCK, MINB) trace_f32_kernel(const TraceParams P)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n = P.n;
    unsigned long long n_items = (unsigned long long)n;
    if (P.n_dev && *P.n_dev < n_items)
        n_items = *P.n_dev;
    // zone phase: n0 entries from the FP32 phase; re-queueing needs them all
    // in the ring (with one entry per geodesic the ring cannot overflow; the
    // check stays as a guard)
    unsigned long long n0 = 0;
    bool requeue = false;
    if (PHASE != 0) {
        const unsigned long long zc = *P.zcount;
        const unsigned long long cap = (unsigned long long)P.zcap;
        n0 = zc < cap ? zc : cap;
        requeue = P.zone_quantum > 0 && zc <= cap && P.zpush != nullptr;
    }
    const unsigned long long zcap = (unsigned long long)P.zcap;
    const bool can_defer = PHASE == 0 && P.zbuf != nullptr && P.fp64_zone > 0.0;
    const float tol = (float)P.tol;
    const float h0 = (float)P.h0;
    // zone phase: re-queueing is tested every zone_quantum iterations of a
    // warp, staggered over the warps of the grid, so that the warps do not
    // all reach the queue's counters at once
    const uint32_t zq = P.zone_quantum > 0 ? (uint32_t)P.zone_quantum : 1u;
    const uint32_t zq_min = zq > 1 ? zq / 2 : 1u;
    uint32_t wit = (uint32_t)((blockIdx.x * (unsigned)(BLOCK / 32) + (threadIdx.x >> 5)) % zq);

    bool has = false, drained = false, timed_out = false;
    int64_t id = 0;
    RayConst rc;
    if (TEAM)
        rc = RayConst{};     // a helper lane passes its (unused) constants along
    // TEAM: the warp is in the phase's tail (warp-uniform, set once)
    bool tail = false;
    uint32_t tcheck = 0;
    const unsigned long long lanes_total = (unsigned long long)gridDim.x * BLOCK;
    float y[8], c[8];
    float h = 0.f, rnow = 0.f;
    uint32_t nsteps = 0, quantum = 0;
    int since_renorm = 0;
    // FP64 zone phase: (y, c) hold the FP64 state's bit patterns (see
    // d_from_bits) instead of an FP32 pair while a geodesic is in the zone
    bool zd = false;
    auto to_pair = [&]() {
        if (PHASE == 1 && zd) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                zsplit(d_from_bits(y[i], c[i]), y[i], c[i]);
            zd = false;
        }
    };
    Counters C;
    const unsigned long long t_start = global_ns();
    uint32_t iter = 0;

    for (;;) {
        // ---- refill idle lanes from the queue (one atomic per warp); in the
        // tail of a TEAM zone phase up to 16 geodesics per warp
        unsigned need = __ballot_sync(FULL, !has);
        if (TEAM && tail)
            need = low_bits(need, __popc(need) > 16 ? __popc(need) - 16 : 0);
        bool empty = false;
        if (need && !drained) {
            unsigned long long my = 0;
            bool got = false;
            if (PHASE != 0) {
                unsigned take = 0;
                const unsigned long long base = warp_claim_queue(
                    P.zhead, n0, requeue ? P.zpush : nullptr, need, &take, &empty);
                const unsigned rank = __popc(need & lt_mask);
                my = base + rank;
                got = ((need >> lane) & 1u) && rank < take;
            } else {
                const unsigned long long base = warp_claim(P.head, need);
                if (base + __popc(need) >= n_items)
                    drained = true;
                my = base + __popc(need & lt_mask);
                got = !has && my < n_items;
            }
            if (got) {
                bool go = true;
                if (PHASE != 0) {
                    ZoneEntry &e = P.zbuf[my % zcap];
                    go = wait_seq(&e.seq, (uint32_t)(my + 1ull));
                    if (go) {
                        // read past L1: the slot may have been read here before
                        const float4 *v = reinterpret_cast<const float4 *>(e.y);
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const float4 a4 = __ldcg(v + q), c4 = __ldcg(v + 2 + q);
                            y[4 * q] = a4.x;
                            y[4 * q + 1] = a4.y;
                            y[4 * q + 2] = a4.z;
                            y[4 * q + 3] = a4.w;
                            c[4 * q] = c4.x;
                            c[4 * q + 1] = c4.y;
                            c[4 * q + 2] = c4.z;
                            c[4 * q + 3] = c4.w;
                        }
                        id = (int64_t)__ldcg(reinterpret_cast<const long long *>(&e.id));
                        h = __ldcg(&e.h);
                        rnow = __ldcg(&e.rnow);
                        nsteps = __ldcg(&e.nsteps);
                        since_renorm = __ldcg(&e.since_renorm);
                        zd = PHASE == 1 && __ldcg(&e.fmt) == ZE_FP64;
                        st_release(&e.seq, 0u);
                        load_const_full(P, id, rc);
                        quantum = 0;
                    } else {
                        C.status(ST_NONE);   // hand-over timed out (counted, never expected)
                    }
                } else {
                    id = (int64_t)my;
                    go = P.status[id] == ST_NONE;     // set-up already ended it
                    if (go) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            y[i] = P.s_state[i * n + id];
                            c[i] = P.s_state[(8 + i) * n + id];
                        }
                        if (P.renorm_every > 0)
                            load_const_full(P, id, rc);   // FP64 spin for re-solving k^t
                        else
                            load_const_f32(P, id, rc);
                        h = h0;
                        nsteps = 0;
                        since_renorm = 0;
                        rnow = ks_r(rc.af * rc.af, y[1], y[2], y[3]);
                    }
                }
                if (go) {
                    if (timed_out) {
                        P.status[id] = ST_TIMEOUT;
                        P.steps[id] = nsteps;
                        C.status(ST_TIMEOUT);
                        if (PHASE != 0) {
                            to_pair();
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                P.s_state[i * n + id] = y[i];
                                P.s_state[(8 + i) * n + id] = c[i];
                            }
                        }
                    } else {
                        has = true;
                    }
                }
            }
        }
        if (!__any_sync(FULL, has)) {
            // warp-uniform: drained / empty come from the shuffled claim
            if (PHASE != 0 ? empty : drained)
                break;
            continue;
        }
        // ---- zone entries: defer them to the zone phase (PHASE 0)
        bool in_zone = has && rnow < rc.zonef;
        if (can_defer) {
            const unsigned dm = __ballot_sync(FULL, in_zone && !timed_out);
            if (dm) {
                const unsigned long long zb = warp_claim(P.zcount, dm);
                if ((dm >> lane) & 1u) {
                    const unsigned long long slot = zb + __popc(dm & lt_mask);
                    if (slot < zcap) {
                        ZoneEntry &e = P.zbuf[slot];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            e.y[i] = y[i];
                            e.c[i] = c[i];
                        }
                        e.id = id;
                        e.h = h;
                        e.rnow = rnow;
                        e.nsteps = nsteps;
                        e.since_renorm = since_renorm;
                        e.fmt = ZE_PAIR;
                        e.seq = (uint32_t)(slot + 1ull);   // visible to the next launch
                        ++C.def;
                        has = false;
                        in_zone = false;
                    }
                }
            }
        }
        // clipping deferred to the clip pass: the last step ran in FP32 (front
        // of the clip queue) or in the zone's arithmetic (back)
        bool pend32 = false, pend64 = false, clip_bits = false;
        // ---- TEAM tail: each geodesic taking a zone attempt gets an idle
        // lane of its warp as helper, if there are enough (warp-uniform)
        // a zone attempt's result into the lane: step length, r, status, the
        // deferred clip, and the state -- FP64 bits while the geodesic stays
        // in the zone, the FP32 pair once it leaves it
        auto apply_zone = [&](const ZoneResultD &R, int &st_out, ClipRec &cr_out) {
            h = R.h;
            rnow = R.rnow;
            since_renorm = R.since_renorm;
            st_out = R.st;
            cr_out = R.clip;
            C.rhs64 += R.nrhs;
            C.acc += R.nacc;
            ++C.att64;
            if (R.st == ST_NONE && !(rnow < rc.zonef)) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    zsplit(R.y.v[i], y[i], c[i]);
                zd = false;
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    d_to_bits(R.y.v[i], y[i], c[i]);
            }
        };
        int team_st = ST_NONE;
        ClipRec team_cr;
        bool team_owner = false, fin = false;
        if (TEAM && PHASE == 1 && tail) {
            const bool zstep = has && in_zone && !timed_out && (int64_t)nsteps < P.max_steps;
            const unsigned own = __ballot_sync(FULL, zstep);
            const unsigned idl = __ballot_sync(FULL, !has);
            const int no = __popc(own);
            if (no > 0 && __popc(idl) >= no) {
                const unsigned helpers = low_bits(idl, no);
                const unsigned tmask = own | helpers;
                const bool is_helper = (helpers >> lane) & 1u;
                if (zstep || is_helper) {
                    const int partner = zstep ? nth_bit(helpers, __popc(own & lt_mask))
                                              : nth_bit(own, __popc(helpers & lt_mask));
                    Y8d ys;
                    if (zstep) {
                        if (!zd) {
#pragma unroll
                            for (int i = 0; i < 8; ++i)
                                d_to_bits((double)y[i] + (double)c[i], y[i], c[i]);
                            zd = true;
                        }
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            ys.v[i] = d_from_bits(y[i], c[i]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            ys.v[i] = 0.0;
                    }
                    const ZoneResultD R = zone_step_team<RM>(rc, P, id, ys, h, rnow,
                                                             since_renorm, is_helper, partner,
                                                             tmask);
                    if (zstep)
                        apply_zone(R, team_st, team_cr);
                    team_owner = zstep;
                }
            }
        }
        if (has) {
            int st = ST_NONE;
            ClipRec cr;
            bool zone_step_taken = false;
            if (timed_out) {
                st = ST_TIMEOUT;
            } else if ((int64_t)nsteps >= P.max_steps) {
                st = ST_MAXSTEPS;
            } else {
                ++nsteps;
                ++quantum;
                ++C.att;
                if (PHASE == 1 && in_zone) {
                    // FP64 zone phase: the state stays FP64 from one attempt
                    // to the next
                    if (TEAM && team_owner) {
                        st = team_st;            // taken with a helper above
                        cr = team_cr;
                    } else {
                        if (!zd) {
#pragma unroll
                            for (int i = 0; i < 8; ++i)
                                d_to_bits((double)y[i] + (double)c[i], y[i], c[i]);
                            zd = true;
                        }
                        Y8d ys;
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            ys.v[i] = d_from_bits(y[i], c[i]);
                        apply_zone(zone_step_d<RM>(rc, P, id, ys, h, rnow, since_renorm), st, cr);
                    }
                    zone_step_taken = true;
                } else if (PHASE == 2 && in_zone) {
                    LaneF ls;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        ls.y[i] = y[i];
                        ls.c[i] = c[i];
                    }
                    ls.h = h;
                    ls.rnow = rnow;
                    // float-float zone phase
                    const ZoneResult R = zone_step_df<RM>(rc, P, id, ls, since_renorm);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        y[i] = R.s.y[i];
                        c[i] = R.s.c[i];
                    }
                    h = R.s.h;
                    rnow = R.s.rnow;
                    since_renorm = R.since_renorm;
                    st = R.st;
                    cr = R.clip;
                    zone_step_taken = true;
                    C.rhs64 += R.nrhs;
                    C.acc += R.nacc;
                    ++C.att64;
                } else {
                    // (stepping phase: a geodesic inside the zone is always
                    // deferred -- the zone buffer holds one entry per geodesic;
                    // one that could not be would be counted and step in FP32)
                    if (PHASE == 0 && in_zone)
                        C.status(ST_NONE);
                    uint32_t r = 0;
                    // FP32 steps: the variant's right-hand-side mode in the
                    // stepping phase; out of line in the zone phase (as in the
                    // default stepping variant, so that a geodesic's FP32
                    // steps are the same arithmetic in either launch)
                    st = step_once<true, float, false, PHASE == 0 ? RM : RHS_CALL>(
                        rc, P, id, tol, y, c, h, rnow, r, C.acc, since_renorm, nullptr,
                        P.clipq ? &cr : nullptr);
                    C.rhs32 += r;
                    if (PHASE != 0) {
                        C.r32z += r;
                        ++C.a32z;
                    }
                }
            }
            // a deferred clip of an FP64 zone-phase step keeps the FP64 state
            // before the step, exactly (flagged in the clip queue)
            clip_bits = st != ST_NONE && zd && cr.pending && zone_step_taken;
            if (st != ST_NONE) {
                if (!clip_bits)
                    to_pair();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    P.s_state[i * n + id] = y[i];
                    P.s_state[(8 + i) * n + id] = c[i];
                }
                P.status[id] = st;
                P.steps[id] = (int32_t)nsteps;
                if (cr.pending) {
                    P.clip_h[id] = h;
                    P.clip_shi[id] = cr.s_hi;
                    pend64 = zone_step_taken;
                    pend32 = !zone_step_taken;
                }
                C.status(st);
                has = false;
                fin = true;
            }
        }
        if (P.clipq)
            enqueue_clips(P, pend32, pend64, id, clip_bits);
        // ---- TEAM: count the phase's finished geodesics; a warp enters the
        // tail once at most half as many remain as the grid has lanes
        if (TEAM && PHASE == 1) {
            const unsigned fm = __ballot_sync(FULL, fin);
            if (fm && lane == __ffs(fm) - 1)
                atomicAdd(P.zdone, (unsigned long long)__popc(fm));
            if (!tail && ((++tcheck & 7u) == 0u)) {
                int t = 0;
                if (lane == 0) {
                    const unsigned long long done = ld_relaxed(P.zdone);
                    t = 2ull * (n0 - (done < n0 ? done : n0)) <= lanes_total ? 1 : 0;
                }
                tail = __shfl_sync(FULL, t, 0) != 0;
            }
        }
        // ---- zone phase: every zone_quantum iterations of the warp, a
        // geodesic that took at least half a quantum of attempts yields its
        // lane to one that waits in the queue (processor sharing), so that
        // the phase is not left with a second, partly filled wave of lanes.
        // The re-queue points of the warps are staggered: when all warps
        // reached the queue counters' compare-and-swap together, each
        // re-queue point cost a warp ~150 us of retries (measured on the
        // 1024 x 1024 image), several attempts' worth.
        // TEAM tail: a warp keeps at most 16 geodesics, the others go back to
        // the queue for warps with room (no processor sharing any more)
        bool rq_point = false, want = false, force = false;
        if (PHASE != 0 && requeue) {
            if (TEAM && tail) {
                const unsigned hm = __ballot_sync(FULL, has);
                want = has && !timed_out && __popc(hm & lt_mask) >= 16;
                rq_point = force = true;
            } else if (++wit >= zq) {
                wit = 0;
                want = has && !timed_out && quantum >= zq_min;
                rq_point = true;
            }
        }
        if (rq_point) {
            const unsigned pm = __ballot_sync(FULL, want);
            if (pm) {
                const int leader = __ffs(pm) - 1;
                int waiting = 0;
                if (lane == leader)
                    waiting = force || n0 + ld_relaxed(P.zpush) > ld_relaxed(P.zhead) ? 1 : 0;
                waiting = __shfl_sync(FULL, waiting, leader);
                if (waiting) {
                    const unsigned long long b = warp_claim(P.zpush, pm);
                    if (want) {
                        const unsigned long long idx = n0 + b + __popc(pm & lt_mask);
                        ZoneEntry &e = P.zbuf[idx % zcap];
                        if (wait_seq(&e.seq, 0u)) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                e.y[i] = y[i];
                                e.c[i] = c[i];
                            }
                            e.id = id;
                            e.h = h;
                            e.rnow = rnow;
                            e.nsteps = nsteps;
                            e.since_renorm = since_renorm;
                            e.fmt = zd ? ZE_FP64 : ZE_PAIR;
                            st_release(&e.seq, (uint32_t)(idx + 1ull));
                            ++C.req;
                            has = false;
                        } else {
                            C.status(ST_NONE);   // slot never freed (counted, never expected)
                            quantum = 0;
                        }
                    }
                }
            }
        }
        // ---- wall-time budget or abort flag (warp-uniform decision)
        if ((P.budget_ns || P.abort) && ((++iter & 31u) == 0) && !timed_out) {
            bool over = false;
            if (lane == 0)
                over = stop_requested(P, t_start);
            timed_out = __shfl_sync(FULL, over, 0);
        }
    }
    C.flush(P.stats);
}

#endif // KERR_TYPES_ONLY

} // namespace kerr
