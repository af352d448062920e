// kerr_fixed.cu -- paper-mode integration: every geodesic takes exactly
// `nsteps` classic RK4 steps of fixed length h (Sec. 3), with no error
// control and no termination test -- the setting in which the paper times
// its kernels (Sec. 4.2, Tables 2-3: time per RK4 step per ray).  State in
// registers, one geodesic per thread; the state array is read once and
// written once per launch, in SoA ([8][n]) or AoS ([n][8]) layout.
#include "kerr_trace.cuh"
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

template <typename T, bool AOS>
cudaError_t launch(void *state, int64_t n, int nsteps, double h, double a, cudaStream_t s)
{
    const int64_t blocks = (n + 127) / 128;
    rk4_fixed_kernel<T, AOS><<<(unsigned)blocks, 128, 0, s>>>(static_cast<T *>(state), n,
                                                              nsteps, (T)h, (T)a);
    return cudaGetLastError();
}

} // namespace

extern "C" int kerr_rk4_fixed(double a, int32_t fp64, int32_t layout, void *state, int64_t n,
                              int32_t nsteps, double h, void *stream)
{
    if (!(std::fabs(a) <= 1.0) || (fp64 != 0 && fp64 != 1) ||
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
    cudaError_t e;
    if (fp64)
        e = layout == KERR_LAYOUT_AOS ? launch<double, true>(state, n, nsteps, h, a, s)
                                      : launch<double, false>(state, n, nsteps, h, a, s);
    else
        e = layout == KERR_LAYOUT_AOS ? launch<float, true>(state, n, nsteps, h, a, s)
                                      : launch<float, false>(state, n, nsteps, h, a, s);
    if (e != cudaSuccess)
        return kerr::kerr_set_error(KERR_ECUDA, cudaGetErrorString(e));
    return KERR_OK;
}
