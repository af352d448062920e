// FP32+Kahan path: the stepping phase with two geodesics per thread
// (variants 10-13; its own translation unit so that it compiles in parallel).
#include "kerr_trace_x2.cuh"
#include "kerr_variants.h"

namespace kerr {

template <int B, int M>
static cudaError_t launch_x2(const TraceParams &P, int sms, cudaStream_t s)
{
    int per_sm = 0;
    const cudaError_t eo = blocks_per_sm((const void *)trace_f32x2_kernel<B, M>, B, &per_sm);
    if (eo != cudaSuccess)
        return eo;
    long long grid = (long long)per_sm * sms;
    const long long need = (P.n + 2LL * B - 1) / (2LL * B);   // two geodesics per thread
    if (need < grid)
        grid = need < 1 ? 1 : need;
    trace_f32x2_kernel<B, M><<<(unsigned)grid, B, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_trace_f32x2(const TraceParams &P, int v, int sms, cudaStream_t s)
{
    switch (v) {
#define KERR_CASE(i, b, m) \
    case i:                \
        return launch_x2<b, m>(P, sms, s);
        KERR_VARIANT_LIST_X2(KERR_CASE)
#undef KERR_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

} // namespace kerr
