// kerr_df.cuh -- float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  GB300 executes FP64 at a small fraction of its
// FP32 rate, so the steps inside the FP64 zone can use this type instead of
// double: same integrator code (it is templated on the number type), ~48-bit
// precision, FP32-pipe throughput.
//
// Building blocks (published error-free transformations):
//   two_sum        Knuth's TwoSum: s + e = a + b exactly.
//   quick_two_sum  Dekker's Fast2Sum (|a| >= |b|).
//   two_prod       Dekker's product with a fused multiply-add: p + e = a b.
// On top of them: addition with one TwoSum on the high parts (error bounded by
// ~2^-44 (|x| + |y|)), multiplication via two_prod, and reciprocal, square
// root and reciprocal square root as one Newton correction of the hardware
// approximation of the high part.
#pragma once

#include "kerr_math.cuh"

namespace kerr {

// The dfloat overloads below would hide the float/double versions inside this
// namespace; bring those into the overload set.
using ::fabs;
using ::fmax;
using ::fmin;
using ::isfinite;

struct dfloat {
    float hi, lo;
    __device__ __forceinline__ dfloat() : hi(0.f), lo(0.f) {}
    __device__ __forceinline__ dfloat(float h, float l) : hi(h), lo(l) {}
    // from a double constant (compile-time literals in the templated code)
    __device__ __forceinline__ explicit dfloat(double d)
    {
        hi = (float)d;
        lo = (float)(d - (double)hi);
    }
    __device__ __forceinline__ explicit dfloat(float f) : hi(f), lo(0.f) {}
    __device__ __forceinline__ explicit dfloat(int i) : hi((float)i), lo(0.f) {}
};

// accel<dfloat> keeps the explicit vector e (see FoldE)
template <> struct FoldE<dfloat> {
    static constexpr bool value = false;
};

__device__ __forceinline__ dfloat quick_two_sum(float a, float b)
{
    const float s = a + b;
    return dfloat(s, b - (s - a));
}

__device__ __forceinline__ dfloat two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return dfloat(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ dfloat two_prod(float a, float b)
{
    const float p = a * b;
    return dfloat(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y)
{
    dfloat s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }

__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y)
{
    dfloat p = two_prod(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.lo, p.lo);
    e = __fmaf_rn(x.lo, y.hi, e);
    return quick_two_sum(p.hi, e);
}

__device__ __forceinline__ dfloat k_rcp(dfloat x)
{
    const float r0 = k_rcp(x.hi);
    // e = 1 - x r0 (exact enough: two_prod keeps the rounding error of x.hi r0)
    const dfloat xr = x * dfloat(r0, 0.f);
    const float e = (1.0f - xr.hi) - xr.lo;
    return quick_two_sum(r0, r0 * e);
}

__device__ __forceinline__ dfloat operator/(dfloat x, dfloat y) { return x * k_rcp(y); }

__device__ __forceinline__ dfloat k_sqrt(dfloat x)
{
    if (!(x.hi > 0.f))
        return dfloat(x.hi == 0.f ? 0.f : __int_as_float(0x7fc00000), 0.f);
    const float s0 = k_sqrt(x.hi);
    const dfloat s2 = two_prod(s0, s0);
    const float r = ((x.hi - s2.hi) - s2.lo) + x.lo;      // x - s0^2
    return quick_two_sum(s0, r * (0.5f * k_rcp(s0)));
}

__device__ __forceinline__ dfloat k_rsqrt(dfloat x)
{
    const float y0 = k_rsqrt(x.hi);
    // y = y0 + y0 (1 - x y0^2) / 2
    const dfloat y2 = two_prod(y0, y0);
    const dfloat xy2 = x * y2;
    const float e = (1.0f - xy2.hi) - xy2.lo;
    return quick_two_sum(y0, 0.5f * y0 * e);
}

__device__ __forceinline__ dfloat k_fma(dfloat a, dfloat b, dfloat c) { return a * b + c; }

__device__ __forceinline__ void recip2(dfloat p, dfloat q, dfloat &ip, dfloat &iq)
{
    ip = k_rcp(p);
    iq = k_rcp(q);
}

__device__ __forceinline__ bool operator<(dfloat x, dfloat y)
{
    return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo);
}
__device__ __forceinline__ bool operator>(dfloat x, dfloat y) { return y < x; }
__device__ __forceinline__ bool operator<=(dfloat x, dfloat y) { return !(y < x) && x.hi == x.hi && y.hi == y.hi; }
__device__ __forceinline__ bool operator>=(dfloat x, dfloat y) { return y <= x; }
__device__ __forceinline__ bool operator==(dfloat x, dfloat y) { return x.hi == y.hi && x.lo == y.lo; }
__device__ __forceinline__ bool operator!=(dfloat x, dfloat y) { return !(x == y); }

__device__ __forceinline__ dfloat fabs(dfloat x) { return x.hi < 0.f ? -x : x; }
__device__ __forceinline__ dfloat fmax(dfloat x, dfloat y) { return (x < y) ? y : x; }
__device__ __forceinline__ dfloat k_absmax(dfloat u, dfloat v) { return fmax(fabs(u), fabs(v)); }
__device__ __forceinline__ dfloat fmin(dfloat x, dfloat y) { return (y < x) ? y : x; }
__device__ __forceinline__ bool isfinite(dfloat x) { return ::isfinite(x.hi) && ::isfinite(x.lo); }
__device__ __forceinline__ bool k_isfinite(dfloat x) { return isfinite(x); }

__device__ __forceinline__ dfloat &operator+=(dfloat &x, dfloat y) { return x = x + y; }
__device__ __forceinline__ dfloat &operator*=(dfloat &x, dfloat y) { return x = x * y; }

// Step-size factor of the controller evaluated on the high part (the factor
// only scales the next trial step).
__device__ __forceinline__ dfloat step_factor(dfloat err)
{
    if (!isfinite(err))
        return dfloat(0.2f);
    if (err.hi == 0.f)
        return dfloat(5.0f);
    const float f = 0.9f * exp2f(-0.2f * __log2f(err.hi));
    return dfloat(fminf(5.0f, fmaxf(0.2f, f)));
}

} // namespace kerr
