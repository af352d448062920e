// kerr_math.cuh -- device arithmetic of the Cartesian Kerr-Schild geodesic
// integrator (arXiv:1706.07062, Sec. 2.1).  Units G = c = M = 1.
//
// State of one geodesic: y = (t, x, y, z, k^t, k^x, k^y, k^z), k = dx/dlambda.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace kerr {

// ---------------------------------------------------------------------------
// Precision-specific primitives.  FP32 uses the hardware approximations of
// the PTX ISA (rcp/rsqrt/sqrt .approx, relative error ~2^-23).  FP64 refines
// the PTX ISA's approximate FP64 reciprocal and reciprocal square root by one
// higher-order Newton-Raphson step (Markstein-style refinement: with
// e = 1 - x y0 for 1/x, or e = 1 - x y0^2 for 1/sqrt(x), the series
// y0 (1 + e + e^2) and y0 (1 + e/2 + 3e^2/8) leave an error of order e^3),
// and takes sqrt(v) as v rsqrt(v) plus one residual correction
// s + (v - s^2) rsqrt(v) / 2.  On GB300 FP64 runs at 1/64 of the FP32 rate,
// and these take about a third of the FP64 instructions of the correctly
// rounded operators; their error stays within a few units in the last place
// (tested against 1/x, 1/sqrt(x) and sqrt(x) on the device).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float k_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float k_rsqrt(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float k_sqrt(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double k_rcp(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = __fma_rn(-x, y, 1.0);
    return __fma_rn(y, __fma_rn(e, e, e), y);
}
__device__ __forceinline__ double k_rsqrt(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = __fma_rn(-(x * y), y, 1.0);
    return __fma_rn(y * e, __fma_rn(0.375, e, 0.5), y);
}
__device__ __forceinline__ double k_sqrt(double v)
{
    const double y = k_rsqrt(v);
    const double s = v * y;
    const double r = __fma_rn(-s, s, v);
    const double q = __fma_rn(r, 0.5 * y, s);
    return v == 0.0 ? v : q;          // sqrt(+-0) = +-0 (v y would be NaN)
}

// The square root inside the right-hand side.  FP64: v rsqrt(v) without the
// residual correction of k_sqrt (within ~2 ulp instead of ~1; the argument
// d^2 + 4 a^2 z^2 is positive away from the ring singularity, so no zero
// guard): four FP64 instructions fewer per right-hand side.  Other types:
// their k_sqrt.
template <typename T> __device__ __forceinline__ T k_sqrt_rhs(T v) { return k_sqrt(v); }
__device__ __forceinline__ double k_sqrt_rhs(double v) { return v * k_rsqrt(v); }

__device__ __forceinline__ float k_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double k_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// FP64 predicates on the bit pattern, with integer instructions: on GB300 an
// FP64 compare or min/max occupies the FP64 pipe like an FMA (~80 cycles per
// warp instruction), integer instructions do not.
// x is finite (exponent field not all ones).
__device__ __forceinline__ bool k_isfinite(double x)
{
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}
__device__ __forceinline__ bool k_isfinite(float x) { return isfinite(x); }
// max(|u|, |v|): for non-negative IEEE numbers the bit patterns order like
// the values.  A NaN operand gives a NaN (fmax would return the other one).
__device__ __forceinline__ double k_absmax(double u, double v)
{
    const long long m = 0x7fffffffffffffffll;
    const long long a = __double_as_longlong(u) & m, b = __double_as_longlong(v) & m;
    return __longlong_as_double(a > b ? a : b);
}
__device__ __forceinline__ float k_absmax(float u, float v) { return fmaxf(fabsf(u), fabsf(v)); }

// Order tests against a finite v >= 0 on the bit patterns, with integer
// instructions: read as unsigned 64-bit integers, the patterns of the numbers
// >= 0 order like the values, a NaN with the sign bit clear lies above +inf,
// and every pattern with the sign bit set above those.  Each is false for a
// NaN u, as the FP64 comparison is.
__device__ __forceinline__ bool k_le_nonneg(double u, double v)      // u <= v
{
    return (unsigned long long)__double_as_longlong(u) <=
           (unsigned long long)__double_as_longlong(v);
}
__device__ __forceinline__ bool k_lt_nonneg(double u, double v)      // u < v
{
    return (unsigned long long)__double_as_longlong(u) <
           (unsigned long long)__double_as_longlong(v);
}
__device__ __forceinline__ bool k_gt_nonneg(double u, double v)      // u > v
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(u);
    return b > (unsigned long long)__double_as_longlong(v) && b <= 0x7ff0000000000000ull;
}

// Two reciprocals 1/p and 1/q.  FP32: two hardware approximations.  FP64:
// one reciprocal of p q shared by both (p q stays far from overflow for any
// radius below ~1e50).
__device__ __forceinline__ void recip2(float p, float q, float &ip, float &iq)
{
    ip = k_rcp(p);
    iq = k_rcp(q);
}
__device__ __forceinline__ void recip2(double p, double q, double &ip, double &iq)
{
    const double t = k_rcp(p * q);
    ip = q * t;
    iq = p * t;
}

// Kerr-Schild radius from eq. CKSr: the positive root r^2 of
// r^4 - (R^2 - a^2) r^2 - a^2 z^2 = 0.
template <typename T>
__device__ __forceinline__ T ks_r2(T a2, T x, T y, T z)
{
    const T d = k_fma(x, x, k_fma(y, y, z * z)) - a2;
    return T(0.5) * (d + k_sqrt(k_fma(d, d, T(4) * a2 * (z * z))));
}

template <typename T>
__device__ __forceinline__ T ks_r(T a2, T x, T y, T z)
{
    return k_sqrt(ks_r2(a2, x, y, z));
}

// r after an FP64 zone step of the FP32+Kahan path: the right-hand side's
// halved form of eq. CKSr's root, and both roots as v rsqrt(v) without the
// residual correction (within a few ulp; ten FP64 instructions fewer than
// ks_r).  Other types: ks_r.
template <typename T>
__device__ __forceinline__ T ks_r_zone(T a2, T x, T y, T z)
{
    return ks_r(a2, x, y, z);
}
__device__ __forceinline__ double ks_r_zone(double a2, double x, double y, double z)
{
    const double D = 0.5 * k_fma(x, x, k_fma(y, y, k_fma(z, z, -a2)));
    const double r2 = D + k_sqrt_rhs(k_fma(D, D, (a2 * z) * z));
    return r2 * k_rsqrt(r2);
}

// Whether accel<T> folds the vector e of d l into the coefficients of x'' and
// y'' (every type but float-float, which specialises this to false).
template <typename T> struct FoldE {
    static constexpr bool value = true;
};

// ---------------------------------------------------------------------------
// Geodesic acceleration d k^mu / d lambda in the split-metric form of
// Sec. 2.1, eqs. opt0 and opti:
//   x0'' =  k^al D_{0 al} - F,
//   xi'' = -k^al (D_{i al} - D_{al i}/2) + F l^i,
// with D_{be al} = d_al(f l_be l_ga) k^ga = l_be A_al + f L d_al l_be,
//   L = l_ga k^ga,  A_al = (d_al f) L + f (d_al l_ga) k^ga,
// and F = f (l^be k^al - l^al k^be / 2) D_{be al}.  Two exact properties of
// the Kerr-Schild vector (l is null, and l^i d_i l_be = 0: it is an affinely
// parametrised flat-space geodesic) reduce F to -f L^2 (l^i d_i f) / 2.
// The pieces:
//   r from eq. CKSr; d_i r = (f/2) (x, y, z (1 + a^2/r^2));
//   f = 2 r^3 / q, q = r^4 + a^2 z^2;  d_i f = c1 d_i r + g delta_iz with
//     c1 = f (3/r - 2f), g = -2 f a^2 z / q;
//   l_i = (P x + Q y, P y - Q x, z / r), P = r/s, Q = a/s, s = r^2 + a^2;
//   d_al l_i = (d_al r) e_i + M_{al i}, with
//     e = ((x - 2 r l_x) / s, (y - 2 r l_y) / s, -l_z / r),
//     M_{xx} = M_{yy} = P, M_{yx} = -M_{xy} = Q, M_{zz} = 1 / r, others 0.
// Contracted as the equations need them (exact rearrangements):
//   A_al k^al = L (c1 k.grad r + g k_z) + f (k.grad r (e.k) + P (k_x^2 + k_y^2)
//               + k_z^2 / r)                       (M's antisymmetric part drops),
//   l.grad f  = c1 + g l_z                         (l.grad r = 1 here),
//   x_i''     = (L^2/2) d_i f + f L (dL_i - kd_i) + l_i (F - A.k),
//   with dL_i - kd_i = (d_i r)(e.k) - (k.grad r) e_i - 2Q (k_y, -k_x, 0)_i,
// where dL_i = (d_i l_ga) k^ga and kd_i = k^al d_al l_i; d_i f and d_i r are
// expanded in the last line so that neither vector is formed.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void accel(const T a, const T a2, const T x, const T y, const T z,
                                      const T kt, const T kx, const T ky, const T kz, T &at,
                                      T &ax, T &ay, T &az)
{
    // r^2 = D + sqrt(D^2 + a^2 z^2) with D = (x^2 + y^2 + z^2 - a^2) / 2:
    // eq. CKSr's root with the factors 1/2 and 4 taken out (exact scalings)
    const T a2z = a2 * z;
    const T az2 = a2z * z;
    const T D = T(0.5) * k_fma(x, x, k_fma(y, y, k_fma(z, z, -a2)));
    const T r2 = D + k_sqrt_rhs(k_fma(D, D, az2));
    const T ir = k_rsqrt(r2);
    const T r = r2 * ir;
    T iq, is;                                   // 1/q, 1/s
    recip2(k_fma(r2, r2, az2), r2 + a2, iq, is);
    const T hf = r * r2 * iq;                   // f / 2
    const T f = hf + hf;
    const T P = r * is;
    const T Q = a * is;
    const T lx = k_fma(P, x, Q * y);
    const T ly = k_fma(P, y, -(Q * x));
    const T lz = z * ir;
    // The x, y parts of l.k and of (x, y, zt).k are kept apart: e.k is formed
    // from them, and the vector e then enters x'' and y'' only through the
    // coefficients of (x, y) and of (l_x, l_y) (two instructions fewer per
    // right-hand side; float-float keeps the explicit e)
    constexpr bool kFold = FoldE<T>::value;
    T L, Lxy = T(0), Kxy = T(0);
    if constexpr (kFold) {
        Lxy = k_fma(lx, kx, ly * ky);
        L = Lxy + k_fma(lz, kz, kt);
    } else {
        L = k_fma(lx, kx, k_fma(ly, ky, k_fma(lz, kz, kt)));
    }
    // d_i r = (f/2) (x, y, zt)_i and k . grad r
    const T ir2 = ir * ir;
    const T zt = k_fma(a2z, ir2, z);
    T kr;
    if constexpr (kFold) {
        Kxy = k_fma(x, kx, y * ky);
        kr = hf * k_fma(zt, kz, Kxy);
    } else {
        kr = hf * k_fma(x, kx, k_fma(y, ky, zt * kz));
    }
    // d_i f = c1 d_i r + g delta_iz
    const T c1 = f * k_fma(T(3), ir, -(f + f));
    const T g = -(f + f) * a2z * iq;
    // e of d_al l_i = r_al e_i + M_{al i}: e_x = (x - 2 r l_x) / s,
    // e_y = (y - 2 r l_y) / s, e_z = -z / r^2, and e . k
    const T m2r = -(r + r);
    const T ez = -z * ir2;
    T ek, ex = T(0), ey = T(0);
    if constexpr (kFold) {
        ek = k_fma(is, k_fma(m2r, Lxy, Kxy), ez * kz);
    } else {
        ex = is * k_fma(m2r, lx, x);
        ey = is * k_fma(m2r, ly, y);
        ek = k_fma(ex, kx, k_fma(ey, ky, ez * kz));
    }
    // A_al k^al and l . grad f
    const T gk = k_fma(c1, kr, g * kz);
    const T dLk = k_fma(kr, ek, k_fma(P, k_fma(kx, kx, ky * ky), (ir * kz) * kz));
    const T Ak = k_fma(L, gk, f * dLk);
    const T lf = k_fma(g, lz, c1);
    const T L2 = L * L;
    const T hLL = T(0.5) * L2;
    // at = A.k - F with F = -(f/2) L^2 (l.grad f), as one explicit fused
    // multiply-add (so that no compiler contraction can make the scalar and
    // the packed two-per-thread forms round differently)
    at = k_fma(hf * L2, lf, Ak);
    // x_i'' with d_i f and d_i r expanded: (f/2)(L^2 c1/2 + f L e.k)(x, y, zt)_i
    // - f L (k.grad r) e_i - 2 f L Q (k_y, -k_x, 0)_i + (L^2/2) g delta_iz
    // + l_i (F - A.k)
    const T fL = f * L;
    const T FmA = -at;                          // F - A.k, exactly
    const T hw = hf * k_fma(hLL, c1, fL * ek);
    const T fLkr = fL * kr;
    const T fLQ2 = fL * (Q + Q);
    if constexpr (kFold) {
        // -f L (k.grad r) e_i = -fLkr (x_i - 2 r l_i) / s for i = x, y
        const T al = k_fma(-fLkr, is, hw);
        const T be = k_fma(P + P, fLkr, FmA);
        ax = k_fma(x, al, k_fma(lx, be, -(fLQ2 * ky)));
        ay = k_fma(y, al, k_fma(ly, be, fLQ2 * kx));
    } else {
        ax = k_fma(x, hw, k_fma(-fLkr, ex, k_fma(-fLQ2, ky, lx * FmA)));
        ay = k_fma(y, hw, k_fma(-fLkr, ey, k_fma(fLQ2, kx, ly * FmA)));
    }
    az = k_fma(zt, hw, k_fma(-fLkr, ez, k_fma(hLL, g, lz * FmA)));
}

// ---------------------------------------------------------------------------
// Out-of-line right-hand sides.  A kernel that inlines the eleven right-hand
// sides of an attempt outgrows the instruction cache; its steps can call one
// copy instead.  FP64 steps are also latency-bound on GB300 (1/64 of the
// FP32 rate, one or two warps per scheduler): the pair form evaluates two
// independent right-hand sides in one call, interleaved, for
// instruction-level parallelism.  Same arithmetic as accel<T>.
// ---------------------------------------------------------------------------
template <typename T> struct Acc {
    T t, x, y, z;
};
using Acc64 = Acc<double>;
struct Acc64x2 {
    Acc64 p, q;
};

template <typename T>
static __device__ __noinline__ Acc<T> accel_call(const T a, const T a2, const T x, const T y,
                                                 const T z, const T kt, const T kx, const T ky,
                                                 const T kz)
{
    Acc<T> r;
    accel<T>(a, a2, x, y, z, kt, kx, ky, kz, r.t, r.x, r.y, r.z);
    return r;
}

static __device__ __noinline__ Acc64x2 accel_pair(const double a, const double a2,
                                                  const double x1, const double y1,
                                                  const double z1, const double kt1,
                                                  const double kx1, const double ky1,
                                                  const double kz1, const double x2,
                                                  const double y2, const double z2,
                                                  const double kt2, const double kx2,
                                                  const double ky2, const double kz2)
{
    Acc64x2 r;
    accel<double>(a, a2, x1, y1, z1, kt1, kx1, ky1, kz1, r.p.t, r.p.x, r.p.y, r.p.z);
    accel<double>(a, a2, x2, y2, z2, kt2, kx2, ky2, kz2, r.q.t, r.q.x, r.q.y, r.q.z);
    return r;
}

// ---------------------------------------------------------------------------
// FP64 helpers for set-up, renormalisation and diagnostics.
// ---------------------------------------------------------------------------
struct KSPoint {
    double r, f, lx, ly, lz;
};

// r, f and l at a point (eqs. def:CKS, CKSr), with the refined FP64
// reciprocal square root and the shared reciprocal of the right-hand side
// (within a few ulp; IEEE division and square root cost several times as
// many FP64 instructions on GB300).
__device__ __forceinline__ KSPoint ks_point(double a, double x, double y, double z)
{
    KSPoint p;
    const double a2 = a * a;
    const double r2 = ks_r2(a2, x, y, z);
    const double ir = k_rsqrt(r2);
    p.r = r2 * ir;
    double iq, is;
    recip2(k_fma(r2, r2, a2 * (z * z)), r2 + a2, iq, is);
    p.f = 2.0 * p.r * r2 * iq;
    p.lx = (p.r * x + a * y) * is;
    p.ly = (p.r * y - a * x) * is;
    p.lz = z * ir;
    return p;
}

// g_ab k^a k^b = -kt^2 + |k|^2 + f (kt + l.k)^2 for g = eta + f l l (l_0 = 1).
__device__ __forceinline__ double norm2(const KSPoint &p, const double k[4])
{
    const double L = k[0] + p.lx * k[1] + p.ly * k[2] + p.lz * k[3];
    return -k[0] * k[0] + k[1] * k[1] + k[2] * k[2] + k[3] * k[3] + p.f * L * L;
}

// Solve g_ab k^a k^b = target for k^t with the spatial k fixed:
// (f - 1) kt^2 + 2 f s kt + (|k|^2 + f s^2 - target) = 0, s = l_i k^i.
// branch < 0: smaller root; > 0: larger root; 0: root nearest k[0].
// Returns false when there is no real root.
__device__ __forceinline__ bool solve_kt(const KSPoint &p, double k[4], double target, int branch)
{
    const double s = p.lx * k[1] + p.ly * k[2] + p.lz * k[3];
    const double A = p.f - 1.0;
    const double B = 2.0 * p.f * s;
    const double C = k[1] * k[1] + k[2] * k[2] + k[3] * k[3] + p.f * s * s - target;
    const double disc = B * B - 4.0 * A * C;
    if (!(disc >= 0.0) || A == 0.0)
        return false;
    const double q = -0.5 * (B + copysign(k_sqrt(disc), B));
    const double r1 = q * k_rcp(A);
    const double r2 = (q != 0.0) ? C * k_rcp(q) : r1;
    const double lo = fmin(r1, r2), hi = fmax(r1, r2);
    if (branch == 0)
        k[0] = (fabs(lo - k[0]) <= fabs(hi - k[0])) ? lo : hi;
    else
        k[0] = branch < 0 ? lo : hi;
    return true;
}

// Constants of motion at an FP64 state: E = -p_t, L_z = x p_y - y p_x,
// Carter's Q = p_th^2 + cos^2(th) [a^2 (mu^2 - E^2) + L_z^2 / sin^2(th)] with
// mu^2 = -u^2, p_th = cot(th) (x p_x + y p_y) - r sin(th) p_z, cos(th) = z/r,
// and u^2 = g_ab k^a k^b.  p_a = eta_ab k^b + f l_a L.
__device__ __forceinline__ void constants(double a, const double y[8], float out[4])
{
    const KSPoint p = ks_point(a, y[1], y[2], y[3]);
    const double L = y[4] + p.lx * y[5] + p.ly * y[6] + p.lz * y[7];
    const double pt = -y[4] + p.f * L;
    const double px = y[5] + p.f * p.lx * L;
    const double py = y[6] + p.f * p.ly * L;
    const double pz = y[7] + p.f * p.lz * L;
    const double u2 = pt * y[4] + px * y[5] + py * y[6] + pz * y[7];
    const double E = -pt;
    const double Lz = y[1] * py - y[2] * px;
    const double c = p.lz;                      // cos(theta) = z / r
    const double s2 = 1.0 - c * c;
    const double is = k_rsqrt(s2);              // 1 / sin(theta)
    const double s = s2 * is;
    const double pth = (c * is) * (y[1] * px + y[2] * py) - p.r * s * pz;
    const double Q = pth * pth + c * c * (a * a * (-u2 - E * E) + Lz * Lz * (is * is));
    out[0] = (float)E;
    out[1] = (float)Lz;
    out[2] = (float)Q;
    out[3] = (float)u2;
}

} // namespace kerr
