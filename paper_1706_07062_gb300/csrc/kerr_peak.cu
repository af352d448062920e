// kerr_peak.cu -- fused multiply-add chains that keep the FP32 or FP64 pipe
// of every SM busy: the denominator of the integrator's ALU roofline is this
// GPU's measured rate rather than a datasheet number.
//
// Each thread runs kChains independent chains a <- a m + c (|m| < 1, so the
// values stay bounded) for `iters` rounds, unrolled so that loop control is a
// few percent of the issued instructions; the chains are independent, so the
// rate is set by the pipe's throughput, not by its latency.  The result is
// stored only under a condition the compiler cannot decide, which keeps the
// arithmetic alive without memory traffic.
#include <cuda_runtime.h>

#include "kerr.h"
#include "kerr_f2.cuh"
#include "kerr_variants.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kBlock = 256;

template <typename T> __device__ __forceinline__ T fma_op(T a, T b, T c);
template <> __device__ __forceinline__ float fma_op(float a, float b, float c)
{
    return __fmaf_rn(a, b, c);
}
template <> __device__ __forceinline__ double fma_op(double a, double b, double c)
{
    return __fma_rn(a, b, c);
}
template <> __device__ __forceinline__ float2 fma_op(float2 a, float2 b, float2 c)
{
    return __ffma2_rn(a, b, c);
}

template <typename T> __device__ __forceinline__ T splat(float v);
template <> __device__ __forceinline__ float splat(float v) { return v; }
template <> __device__ __forceinline__ double splat(float v) { return (double)v; }
template <> __device__ __forceinline__ float2 splat(float v) { return make_float2(v, -v); }

__device__ __forceinline__ float first(float v) { return v; }
__device__ __forceinline__ float first(double v) { return (float)v; }
__device__ __forceinline__ float first(float2 v) { return v.x + v.y; }

template <typename T>
__global__ void __launch_bounds__(kBlock) fma_chain_kernel(int64_t rounds, float *sink)
{
    T a[kChains];
    const float t = 1e-3f * (float)threadIdx.x;
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        a[j] = splat<T>(t + (float)j);
    const T m = splat<T>(0.999999f), c = splat<T>(1e-7f);
    for (int64_t i = 0; i < rounds; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int j = 0; j < kChains; ++j)
                a[j] = fma_op(a[j], m, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        s += first(a[j]);
    if (s == -1.2345678f)          // never true for these chains; keeps them alive
        sink[blockIdx.x * kBlock + threadIdx.x] = s;
}

} // namespace

extern "C" int kerr_fma_chain(int32_t kind, int64_t rounds, int32_t blocks_per_sm, float *sink,
                              double *flops, void *stream)
{
    if (kind != KERR_PEAK_FP32 && kind != KERR_PEAK_FP64 && kind != KERR_PEAK_FP32X2)
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_fma_chain: unknown kind");
    if (rounds < 1 || blocks_per_sm < 1 || blocks_per_sm > 8 || !sink)
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_fma_chain: bad arguments");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return kerr::kerr_set_error(KERR_ECUDA, "kerr_fma_chain: no device");
    }
    const int grid = sms * blocks_per_sm;
    cudaStream_t s = (cudaStream_t)stream;
    double per_fma = 2.0;
    if (kind == KERR_PEAK_FP32) {
        fma_chain_kernel<float><<<grid, kBlock, 0, s>>>(rounds, sink);
    } else if (kind == KERR_PEAK_FP64) {
        fma_chain_kernel<double><<<grid, kBlock, 0, s>>>(rounds, sink);
    } else {
        fma_chain_kernel<float2><<<grid, kBlock, 0, s>>>(rounds, sink);
        per_fma = 4.0;                      // two fused multiply-adds per instruction
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return kerr::kerr_set_error(KERR_ECUDA, cudaGetErrorString(e));
    if (flops)
        *flops = per_fma * (double)grid * kBlock * (double)rounds * kUnroll * kChains;
    return KERR_OK;
}
