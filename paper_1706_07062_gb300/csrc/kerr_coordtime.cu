// kerr_coordtime.cu -- geodesics integrated in the coordinate time t
// (Sec. 2.2, eq. geo_t).  State w = (x, y, z, v^x, v^y, v^z), v = dx/dt.
// Along a geodesic k = k^t u with u = (1, v); the affine acceleration
// A(k) = dk/dlambda is quadratic in k and d/dlambda = k^t d/dt, so
//   dx^i/dt = v^i,   dv^i/dt = A^i(u) - v^i A^t(u),
// with A from the split-metric form of eqs. opt0/opti (accel).  This is the
// right-hand side eq. geo_t writes in the split-metric variables.
//
// Step control as in the affine integrator (step doubling, err over the six
// components, the same factor rule); a trial step never passes the end time,
// so the last accepted step lands on it exactly.  Termination after each
// accepted step: captured r < 1.01 r_h, escaped r > r_esc while moving
// outward in the direction of integration, end time reached.
#include "kerr_trace.cuh"
#include "kerr_variants.h"

namespace kerr {
namespace {

template <typename T>
__device__ __forceinline__ void rhs_ct(const T a, const T a2, const T w[6], T dw[6])
{
    T at, ax, ay, az;
    accel<T>(a, a2, w[0], w[1], w[2], T(1), w[3], w[4], w[5], at, ax, ay, az);
    dw[0] = w[3];
    dw[1] = w[4];
    dw[2] = w[5];
    dw[3] = k_fma(-w[3], at, ax);
    dw[4] = k_fma(-w[4], at, ay);
    dw[5] = k_fma(-w[5], at, az);
}

// Increment of one classic RK4 step of length h from w, k1 = rhs(w) given.
template <typename T>
__device__ __forceinline__ void rk4_ct(const T a, const T a2, const T w[6], const T k1[6],
                                       const T h, T d[6])
{
    const T hh = T(0.5) * h;
    T s[6], k2[6], k3[6], k4[6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
        s[i] = k_fma(hh, k1[i], w[i]);
    rhs_ct(a, a2, s, k2);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        s[i] = k_fma(hh, k2[i], w[i]);
    rhs_ct(a, a2, s, k3);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        s[i] = k_fma(h, k3[i], w[i]);
    rhs_ct(a, a2, s, k4);
    const T h6 = h * T(1.0 / 6.0);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        d[i] = h6 * (k1[i] + T(2) * (k2[i] + k3[i]) + k4[i]);
}

template <typename T, bool KAHAN>
__global__ void __launch_bounds__(128) coordtime_kernel(const CoordParams P)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n = P.n;
    const T a = (T)P.a, a2 = a * a;
    const double rh = 1.0 + sqrt(fmax(0.0, 1.0 - P.a * P.a));
    const T rcap = (T)(1.01 * rh);
    const T tol = (T)P.tol;

    bool has = false, drained = false;
    int64_t id = 0;
    T w[6], c[6];
    double t = 0.0, tend = 0.0, dir = 1.0;
    T h = T(0), resc = T(0);
    uint32_t nsteps = 0;
    Counters C;

    for (;;) {
        const unsigned need = __ballot_sync(FULL, !has);
        if (need && !drained) {
            const unsigned long long base = warp_claim(P.head, need);
            if (base + __popc(need) >= (unsigned long long)n)
                drained = true;
            const unsigned long long my = base + __popc(need & lt_mask);
            if (!has && my < (unsigned long long)n) {
                id = (int64_t)my;
                ++C.geo;
                t = P.x0[id];
                double wd[6] = {P.x0[n + id],     P.x0[2 * n + id], P.x0[3 * n + id],
                                P.v0[id],         P.v0[n + id],     P.v0[2 * n + id]};
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    w[i] = (T)wd[i];
                    c[i] = KAHAN ? (T)(wd[i] - (double)w[i]) : T(0);
                }
                tend = P.t_end_each ? P.t_end_each[id] : P.t_end;
                dir = tend >= t ? 1.0 : -1.0;
                h = (T)(dir * P.h0);
                nsteps = 0;
                bool finite = isfinite(t) && isfinite(tend);
#pragma unroll
                for (int i = 0; i < 6; ++i)
                    finite = finite && isfinite(wd[i]);
                const double r0 = finite ? ks_r(P.a * P.a, wd[0], wd[1], wd[2]) : 0.0;
                resc = (T)(P.r_escape > 0.0 ? P.r_escape : (P.r_escape == 0.0 ? r0 : INFINITY));
                int st = ST_NONE;
                if (!finite)
                    st = ST_NONFINITE;
                else if (r0 < 1.01 * rh)
                    st = ST_CAPTURED;
                else if (tend == t)
                    st = ST_ENDTIME;
                if (st != ST_NONE) {
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        P.x_out[(1 + j) * n + id] = wd[j];
                        P.v_out[j * n + id] = wd[3 + j];
                    }
                    P.x_out[id] = t;
                    P.status[id] = st;
                    P.steps[id] = 0;
                    C.status(st);
                } else {
                    has = true;
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
            if ((int64_t)nsteps >= P.max_steps) {
                st = ST_MAXSTEPS;
            } else {
                ++nsteps;
                ++C.att;
                const bool last = dir * (t + (double)h - tend) >= 0.0;
                const T hs = last ? (T)(tend - t) : h;
                T k1[6], df[6], d1[6], d2[6], wm[6], km[6];
                rhs_ct(a, a2, w, k1);
                rk4_ct(a, a2, w, k1, hs, df);
                rk4_ct(a, a2, w, k1, T(0.5) * hs, d1);
#pragma unroll
                for (int i = 0; i < 6; ++i)
                    wm[i] = w[i] + d1[i];
                rhs_ct(a, a2, wm, km);
                rk4_ct(a, a2, wm, km, T(0.5) * hs, d2);
                T err = T(0);
                T dh[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    dh[i] = d1[i] + d2[i];
                    const T delta = (dh[i] - df[i]) * T(1.0 / 15.0);
                    const T sc = tol * (T(1) + fmax(fabs(w[i]), fabs(w[i] + dh[i])));
                    const T e = fabs(delta) / sc;
                    err = (e <= err) ? err : e;     // NaN propagates
                }
                if (std::is_same<T, float>::value)
                    C.rhs32 += 11;
                else
                    C.rhs64 += 11;
                const T fac = step_factor(err);
                if (!(err <= T(1))) {
                    h = hs * fac;
                } else {
                    ++C.acc;
                    bool finite = true;
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        add_incr<KAHAN>(w[i], c[i], dh[i]);
                        finite = finite && isfinite(w[i]);
                    }
                    t = last ? tend : t + (double)hs;
                    if (!finite) {
                        st = ST_NONFINITE;
                    } else {
                        const T r = ks_r(a2, w[0], w[1], w[2]);
                        const T xv = k_fma(w[0], w[3], k_fma(w[1], w[4], w[2] * w[5]));
                        if (r < rcap)
                            st = ST_CAPTURED;
                        else if (r > resc && T(dir) * xv > T(0))
                            st = ST_ESCAPED;
                        else if (last)
                            st = ST_ENDTIME;
                    }
                    h = (last ? h : hs) * fac;
                }
            }
            if (st != ST_NONE) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    P.x_out[(1 + j) * n + id] = (double)w[j] + (double)c[j];
                    P.v_out[j * n + id] = (double)w[3 + j] + (double)c[3 + j];
                }
                P.x_out[id] = t;
                P.status[id] = st;
                P.steps[id] = (int32_t)nsteps;
                C.status(st);
                has = false;
            }
        }
    }
    C.flush(P.stats);
}

template <typename T, bool KAHAN>
cudaError_t launch(const CoordParams &P, int sms, cudaStream_t s)
{
    int per_sm = 0;
    const cudaError_t eo = blocks_per_sm((const void *)coordtime_kernel<T, KAHAN>, 128, &per_sm);
    if (eo != cudaSuccess)
        return eo;
    long long grid = (long long)per_sm * sms;
    const long long need = (P.n + 127) / 128;
    if (need < grid)
        grid = need < 1 ? 1 : need;
    coordtime_kernel<T, KAHAN><<<(unsigned)grid, 128, 0, s>>>(P);
    return cudaGetLastError();
}

} // namespace

cudaError_t launch_coordtime(const CoordParams &P, int fp32, int sms, cudaStream_t s)
{
    return fp32 ? launch<float, true>(P, sms, s) : launch<double, false>(P, sms, s);
}

} // namespace kerr
