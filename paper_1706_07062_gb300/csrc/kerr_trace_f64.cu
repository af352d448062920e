// FP64 path: one persistent kernel per launch configuration; and the check
// entry point of the FP64 reciprocal / square-root primitives.
#include "kerr_trace.cuh"
#include "kerr_variants.h"
#include "kerr.h"

#include <algorithm>

namespace kerr {

template <int B, int M>
static cudaError_t launch_one(const TraceParams &P, int sms, cudaStream_t s)
{
    int per_sm = 0;
    const cudaError_t eo = blocks_per_sm((const void *)trace_f64_kernel<B, M>, B, &per_sm);
    if (eo != cudaSuccess)
        return eo;
    long long grid = (long long)per_sm * sms;
    const long long need = (P.n + B - 1) / B;
    if (need < grid)
        grid = need < 1 ? 1 : need;
    trace_f64_kernel<B, M><<<(unsigned)grid, B, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_trace_f64(const TraceParams &P, int v, int sms, cudaStream_t s)
{
    switch (v) {
#define KERR_CASE(i, b, m, rm) \
    case i:                    \
        return launch_one<b, m>(P, sms, s);
        KERR_VARIANT_LIST(KERR_CASE)
#undef KERR_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

} // namespace kerr

namespace {

__global__ void fp64_math_kernel(const double *__restrict__ x, int64_t n, double *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        out[i] = kerr::k_rcp(v);
        out[n + i] = kerr::k_rsqrt(v);
        out[2 * n + i] = kerr::k_sqrt(v);
    }
}

} // namespace

extern "C" int kerr_check_fp64_math(const double *x, int64_t n, double *out, void *stream)
{
    if (n < 0 || (n > 0 && (!x || !out)))
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_check_fp64_math: bad arguments");
    if (n == 0)
        return KERR_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    fp64_math_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(x, n, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return kerr::kerr_set_error(KERR_ECUDA, cudaGetErrorString(e));
    return KERR_OK;
}
