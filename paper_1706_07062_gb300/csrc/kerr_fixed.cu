// kerr_fixed.cu -- paper-mode integration: every geodesic takes exactly
// `nsteps` classic RK4 steps of fixed length h (Sec. 3), with no error
// control and no termination test -- the setting in which the paper times
// its kernels (Sec. 4.2, Tables 2-3: time per RK4 step per ray).  State in
// registers, one geodesic per thread; the state array is read once and
// written once per launch, in SoA ([8][n]) or AoS ([n][8]) layout.
#include "kerr_trace.cuh"
#include "kerr_f2.cuh"
#include "kerr_variants.h"
#include "kerr.h"

#include <algorithm>

namespace {

using namespace kerr;

template <typename T> struct Vec2;
template <> struct Vec2<float> {
    using V = float4;   // 4 floats = 16 B
    static constexpr int W = 4;
};
template <> struct Vec2<double> {
    using V = double2;  // 2 doubles = 16 B
    static constexpr int W = 2;
};

template <typename T, bool AOS>
__device__ __forceinline__ void load_state(const T *__restrict__ s, int64_t n, int64_t i, T y[8])
{
    if (AOS) {
        // 16-byte vector loads of the contiguous 8-value record
        using V = typename Vec2<T>::V;
        constexpr int W = Vec2<T>::W;
        const V *p = reinterpret_cast<const V *>(s + 8 * i);
#pragma unroll
        for (int q = 0; q < 8 / W; ++q) {
            const V v = p[q];
            const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int j = 0; j < W; ++j)
                y[W * q + j] = e[j];
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            y[j] = s[j * n + i];
    }
}

template <typename T, bool AOS>
__device__ __forceinline__ void store_state(T *__restrict__ s, int64_t n, int64_t i, const T y[8])
{
    if (AOS) {
        using V = typename Vec2<T>::V;
        constexpr int W = Vec2<T>::W;
        V *p = reinterpret_cast<V *>(s + 8 * i);
#pragma unroll
        for (int q = 0; q < 8 / W; ++q) {
            V v;
            T *e = reinterpret_cast<T *>(&v);
#pragma unroll
            for (int j = 0; j < W; ++j)
                e[j] = y[W * q + j];
            p[q] = v;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            s[j * n + i] = y[j];
    }
}

template <typename T, bool AOS>
__global__ void __launch_bounds__(128) rk4_fixed_kernel(T *__restrict__ state, int64_t n,
                                                        int nsteps, T h, T a)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    T y[8];
    load_state<T, AOS>(state, n, i, y);
    const T a2 = a * a;
#pragma unroll 1
    for (int s = 0; s < nsteps; ++s) {
        T A0[4], d[8];
        rhs<RHS_CALL>(a, a2, y[1], y[2], y[3], y[4], y[5], y[6], y[7], A0);
        rk4_incr<RHS_CALL>(a, a2, y, A0, h, d);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            y[j] = y[j] + d[j];
    }
    store_state<T, AOS>(state, n, i, y);
}

// The same steps for two geodesics per thread on packed FP32 instructions:
// thread i advances geodesics i and i + ceil(n/2) (for odd n the last thread
// repeats geodesic i in its second half and stores it once).
template <bool AOS>
__global__ void __launch_bounds__(128) rk4_fixed_x2_kernel(float *__restrict__ state, int64_t n,
                                                           int nsteps, float h, float a)
{
    const int64_t half = (n + 1) / 2;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= half)
        return;
    const int64_t j = i + half < n ? i + half : i;
    float u[8], w[8];
    load_state<float, AOS>(state, n, i, u);
    load_state<float, AOS>(state, n, j, w);
    f2 y[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
        y[q] = f2(u[q], w[q]);
    const f2 av(a, a), hv(h, h);
    const f2 a2 = av * av;
#pragma unroll 1
    for (int s = 0; s < nsteps; ++s) {
        f2 A0[4], d[8];
        rhs<RHS_CALL>(av, a2, y[1], y[2], y[3], y[4], y[5], y[6], y[7], A0);
        rk4_incr<RHS_CALL>(av, a2, y, A0, hv, d);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            y[q] = y[q] + d[q];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        u[q] = y[q].v.x;
        w[q] = y[q].v.y;
    }
    store_state<float, AOS>(state, n, i, u);
    if (j != i)
        store_state<float, AOS>(state, n, j, w);
}

// ---------------------------------------------------------------------------
// Boyer-Lindquist coordinates (Sec. 2.1, eq. 1), the other chart of the
// paper's timing.  The paper does not print its BL equations; this kernel
// uses the Hamiltonian form of the geodesic equations for the BL metric:
// state (t, r, th, ph, p_t, p_r, p_th, p_ph), H = N / (2 Sigma) with
//   N = Delta p_r^2 + p_th^2 - P^2 / Delta + (L / s - a E s)^2,
//   P = (r^2 + a^2) E - a L,  E = -p_t,  L = p_ph,  s = sin th,
//   Sigma = r^2 + a^2 cos^2 th,  Delta = r^2 - 2 r + a^2,
// dx^mu/dlambda = dH/dp_mu, dp_mu/dlambda = -dH/dx^mu (p_t, p_ph constant):
//   dt/dl  = [P (r^2 + a^2) / Delta + a (L - a E s^2)] / Sigma,
//   dr/dl  = Delta p_r / Sigma,   dth/dl = p_th / Sigma,
//   dph/dl = [a P / Delta + L / s^2 - a E] / Sigma,
//   dp_r/dl  = -[(2r - 2) p_r^2 - (4 r E P Delta - P^2 (2r - 2)) / Delta^2] / (2 Sigma)
//              + N r / Sigma^2,
//   dp_th/dl = (L / s - a E s)(L c / s^2 + a E c) / Sigma - N a^2 c s / Sigma^2.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void bl_rhs(const T a, const T y[8], T dy[8])
{
    const T r = y[1], th = y[2];
    T s, c;
    if constexpr (std::is_same<T, float>::value)
        __sincosf(th, &s, &c);
    else
        sincos(th, &s, &c);
    const T E = -y[4], pr = y[5], pth = y[6], L = y[7];
    const T a2 = a * a, r2 = r * r;
    const T Sig = k_fma(a2, c * c, r2);
    const T Del = r2 - T(2) * r + a2;
    const T iS = k_rcp(Sig), iD = k_rcp(Del), is = k_rcp(s);
    const T P = k_fma(r2 + a2, E, -(a * L));
    const T q = k_fma(L, is, -(a * E * s));          // L / s - a E s
    const T N = k_fma(Del * pr, pr, k_fma(pth, pth, k_fma(-(P * P), iD, q * q)));
    const T dDel = T(2) * r - T(2);
    dy[0] = iS * k_fma(P * (r2 + a2), iD, a * (L - a * E * s * s));
    dy[1] = Del * pr * iS;
    dy[2] = pth * iS;
    dy[3] = iS * k_fma(a * P, iD, k_fma(L, is * is, -(a * E)));
    dy[4] = T(0);
    const T dNr = k_fma(dDel, pr * pr, -(T(4) * r * E * P * Del - P * P * dDel) * iD * iD);
    dy[5] = k_fma(-T(0.5) * iS, dNr, N * r * iS * iS);
    dy[6] = k_fma(q * iS, c * k_fma(L, is * is, a * E), -(N * a2 * c * s * iS * iS));
    dy[7] = T(0);
}

template <typename T, bool AOS>
__global__ void __launch_bounds__(128) rk4_fixed_bl_kernel(T *__restrict__ state, int64_t n,
                                                           int nsteps, T h, T a)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    T y[8];
    load_state<T, AOS>(state, n, i, y);
    const T hh = T(0.5) * h, h6 = h * T(1.0 / 6.0);
#pragma unroll 1
    for (int st = 0; st < nsteps; ++st) {
        T k1[8], k2[8], k3[8], k4[8], u[8];
        bl_rhs(a, y, k1);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            u[j] = k_fma(hh, k1[j], y[j]);
        bl_rhs(a, u, k2);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            u[j] = k_fma(hh, k2[j], y[j]);
        bl_rhs(a, u, k3);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            u[j] = k_fma(h, k3[j], y[j]);
        bl_rhs(a, u, k4);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            y[j] = y[j] + h6 * (k1[j] + T(2) * (k2[j] + k3[j]) + k4[j]);
    }
    store_state<T, AOS>(state, n, i, y);
}

// Distant-observer BL start states of a camera (this reading: observer at
// (r_obs, th = incl, ph = 0, t = 0); photon constants E = 1, L = -alpha sin i,
// Q = beta^2 + cos^2 i (alpha^2 - a^2); p_th = sign(beta) sqrt(Theta(i)),
// Theta = Q - cos^2 i (L^2 / sin^2 i - a^2); p_r < 0 (moving inward) from
// H = 0; p_t = -1), in FP64, stored in T.
template <typename T, bool AOS>
__global__ void bl_camera_kernel(kerr_camera cam, T *__restrict__ state)
{
    const int64_t n = (int64_t)cam.nx * cam.ny;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const int64_t px = i % cam.nx, qy = i / cam.nx;
    const double al = -cam.half_width + (px + 0.5) * 2.0 * cam.half_width / cam.nx;
    const double be = -cam.half_width + (qy + 0.5) * 2.0 * cam.half_width / cam.ny;
    const double a = cam.a, r = cam.r_obs, si = sin(cam.incl), ci = cos(cam.incl);
    const double E = 1.0, L = -al * si;
    const double Q = be * be + ci * ci * (al * al - a * a);
    const double Th = Q - ci * ci * (L * L / (si * si) - a * a * E * E);
    const double pth = (be >= 0.0 ? 1.0 : -1.0) * sqrt(fmax(0.0, Th));
    const double Del = r * r - 2.0 * r + a * a;
    const double P = (r * r + a * a) * E - a * L;
    const double q = L / si - a * E * si;
    // Delta p_r^2 = P^2 / Delta - p_th^2 - q^2
    const double pr2 = (P * P / Del - pth * pth - q * q) / Del;
    const double y[8] = {0.0, r, cam.incl, 0.0, -E, -sqrt(fmax(0.0, pr2)), pth, L};
    T yt[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        yt[j] = (T)y[j];
    store_state<T, AOS>(state, n, i, yt);
}

template <typename T, bool AOS>
cudaError_t launch_bl(void *state, int64_t n, int nsteps, double h, double a, cudaStream_t s)
{
    const int64_t blocks = (n + 127) / 128;
    rk4_fixed_bl_kernel<T, AOS><<<(unsigned)blocks, 128, 0, s>>>(static_cast<T *>(state), n,
                                                                 nsteps, (T)h, (T)a);
    return cudaGetLastError();
}

template <bool AOS>
cudaError_t launch_x2(void *state, int64_t n, int nsteps, double h, double a, cudaStream_t s)
{
    const int64_t blocks = ((n + 1) / 2 + 127) / 128;
    rk4_fixed_x2_kernel<AOS><<<(unsigned)blocks, 128, 0, s>>>(static_cast<float *>(state), n,
                                                             nsteps, (float)h, (float)a);
    return cudaGetLastError();
}

template <typename T, bool AOS>
cudaError_t launch(void *state, int64_t n, int nsteps, double h, double a, cudaStream_t s)
{
    const int64_t blocks = (n + 127) / 128;
    rk4_fixed_kernel<T, AOS><<<(unsigned)blocks, 128, 0, s>>>(static_cast<T *>(state), n,
                                                              nsteps, (T)h, (T)a);
    return cudaGetLastError();
}

} // namespace

static int fixed_common(int coords, double a, int32_t fp64, int32_t layout, void *state,
                        int64_t n, int32_t nsteps, double h, void *stream)
{
    if (!(std::fabs(a) <= 1.0) || fp64 < KERR_FIXED_FP32 || fp64 > KERR_FIXED_FP32X2 ||
        (coords != 0 && fp64 == KERR_FIXED_FP32X2) ||
        (layout != KERR_LAYOUT_SOA && layout != KERR_LAYOUT_AOS) || n < 0 || nsteps < 0 ||
        !std::isfinite(h) || (n > 0 && !state))
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_rk4_fixed: invalid arguments");
    if (layout == KERR_LAYOUT_AOS && (reinterpret_cast<uintptr_t>(state) & 15u))
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_rk4_fixed: AoS state must be 16-byte aligned");
    if (n == 0 || nsteps == 0)
        return KERR_OK;
    if (n > (int64_t)INT32_MAX * 128)
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_rk4_fixed: too many geodesics");
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, state) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_rk4_fixed: state must be device memory");
    }
    const cudaStream_t s = (cudaStream_t)stream;
    const bool aos = layout == KERR_LAYOUT_AOS;
    cudaError_t e;
    if (coords == 0 && fp64 == KERR_FIXED_FP32X2) {
        e = aos ? launch_x2<true>(state, n, nsteps, h, a, s) : launch_x2<false>(state, n, nsteps, h, a, s);
    } else if (coords == 0) {
        if (fp64)
            e = aos ? launch<double, true>(state, n, nsteps, h, a, s)
                    : launch<double, false>(state, n, nsteps, h, a, s);
        else
            e = aos ? launch<float, true>(state, n, nsteps, h, a, s)
                    : launch<float, false>(state, n, nsteps, h, a, s);
    } else {
        if (fp64)
            e = aos ? launch_bl<double, true>(state, n, nsteps, h, a, s)
                    : launch_bl<double, false>(state, n, nsteps, h, a, s);
        else
            e = aos ? launch_bl<float, true>(state, n, nsteps, h, a, s)
                    : launch_bl<float, false>(state, n, nsteps, h, a, s);
    }
    if (e != cudaSuccess)
        return kerr::kerr_set_error(KERR_ECUDA, cudaGetErrorString(e));
    return KERR_OK;
}

extern "C" int kerr_rk4_fixed(double a, int32_t fp64, int32_t layout, void *state, int64_t n,
                              int32_t nsteps, double h, void *stream)
{
    return fixed_common(0, a, fp64, layout, state, n, nsteps, h, stream);
}

extern "C" int kerr_rk4_fixed_bl(double a, int32_t fp64, int32_t layout, void *state, int64_t n,
                                 int32_t nsteps, double h, void *stream)
{
    return fixed_common(1, a, fp64, layout, state, n, nsteps, h, stream);
}

extern "C" int kerr_bl_camera_states(const kerr_camera *cam, int32_t fp64, int32_t layout,
                                     void *state, void *stream)
{
    if (!cam || !state || cam->nx <= 0 || cam->ny <= 0 || !(std::fabs(cam->a) < 1.0) ||
        !(cam->half_width > 0.0) || !(cam->r_obs > 2.0) || !(std::sin(cam->incl) > 0.0) ||
        (fp64 != 0 && fp64 != 1) || (layout != KERR_LAYOUT_SOA && layout != KERR_LAYOUT_AOS))
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_bl_camera_states: invalid arguments");
    if (layout == KERR_LAYOUT_AOS && (reinterpret_cast<uintptr_t>(state) & 15u))
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_bl_camera_states: AoS state must be 16-byte aligned");
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, state) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_bl_camera_states: state must be device memory");
    }
    const int64_t n = (int64_t)cam->nx * cam->ny;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    const cudaStream_t s = (cudaStream_t)stream;
    const bool aos = layout == KERR_LAYOUT_AOS;
    if (fp64) {
        if (aos)
            bl_camera_kernel<double, true><<<blocks, 128, 0, s>>>(*cam, static_cast<double *>(state));
        else
            bl_camera_kernel<double, false><<<blocks, 128, 0, s>>>(*cam, static_cast<double *>(state));
    } else {
        if (aos)
            bl_camera_kernel<float, true><<<blocks, 128, 0, s>>>(*cam, static_cast<float *>(state));
        else
            bl_camera_kernel<float, false><<<blocks, 128, 0, s>>>(*cam, static_cast<float *>(state));
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return kerr::kerr_set_error(KERR_ECUDA, cudaGetErrorString(e));
    return KERR_OK;
}
