// kerr_f2.cuh -- two FP32 geodesics per thread on Blackwell's packed FP32
// instructions.
//
// sm_100-family GPUs (GB300 included) execute a pair of FP32 additions,
// multiplications or fused multiply-adds as one instruction (f32x2).  The
// FP32 datapath is as wide as before, so the peak is unchanged, but a warp
// issues half as many arithmetic instructions for the same work -- the FP32
// integrator is bound by instruction issue, not by the FMA pipe.  `f2` holds
// the same quantity of two independent geodesics; instantiating the templated
// right-hand side and RK4 step with T = f2 advances both at once.  Every
// operation is the IEEE round-to-nearest FP32 operation of the scalar code
// (no contraction across operations); square roots and reciprocals have no
// packed form and run per component.
#pragma once

#include "kerr_math.cuh"

namespace kerr {

struct f2 {
    float2 v;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ f2(float2 a) : v(a) {}
    __device__ __forceinline__ f2(float x, float y) : v(make_float2(x, y)) {}
    // broadcast constants (the templated code writes T(0.5), T(3), ...)
    __device__ __forceinline__ explicit f2(double d) : v(make_float2((float)d, (float)d)) {}
    __device__ __forceinline__ explicit f2(int i) : v(make_float2((float)i, (float)i)) {}
};

__device__ __forceinline__ f2 operator+(f2 x, f2 y) { return f2(__fadd2_rn(x.v, y.v)); }
__device__ __forceinline__ f2 operator*(f2 x, f2 y) { return f2(__fmul2_rn(x.v, y.v)); }
// x - y as fma(y, -1, x): the product is exact, so this is one correctly
// rounded subtraction in a single packed instruction
__device__ __forceinline__ f2 operator-(f2 x, f2 y)
{
    return f2(__ffma2_rn(y.v, make_float2(-1.f, -1.f), x.v));
}
__device__ __forceinline__ f2 operator-(f2 x) { return f2(__fmul2_rn(x.v, make_float2(-1.f, -1.f))); }
__device__ __forceinline__ f2 k_fma(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }

__device__ __forceinline__ f2 k_sqrt(f2 x) { return f2(k_sqrt(x.v.x), k_sqrt(x.v.y)); }
__device__ __forceinline__ f2 k_rsqrt(f2 x) { return f2(k_rsqrt(x.v.x), k_rsqrt(x.v.y)); }
__device__ __forceinline__ f2 k_rcp(f2 x) { return f2(k_rcp(x.v.x), k_rcp(x.v.y)); }
__device__ __forceinline__ void recip2(f2 p, f2 q, f2 &ip, f2 &iq)
{
    ip = k_rcp(p);
    iq = k_rcp(q);
}

} // namespace kerr
