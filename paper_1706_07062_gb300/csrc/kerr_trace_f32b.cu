// FP32+Kahan path: stepping-kernel launch configurations 5-9 (compiled apart
// from 0-4 so that the two halves build in parallel).
#include "kerr_trace.cuh"
#include "kerr_variants.h"

namespace kerr {

template <int PH, int B, int M, int RM>
static cudaError_t launch_one(const TraceParams &P, int sms, cudaStream_t s, bool clamp_to_n)
{
    int per_sm = 0;
    const cudaError_t eo = blocks_per_sm((const void *)trace_f32_kernel<PH, B, M, RM>, B, &per_sm);
    if (eo != cudaSuccess)
        return eo;
    long long grid = (long long)per_sm * sms;
    const long long need = (P.n + B - 1) / B;
    if (clamp_to_n && need < grid)
        grid = need < 1 ? 1 : need;
    trace_f32_kernel<PH, B, M, RM><<<(unsigned)grid, B, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_trace_f32_hi(const TraceParams &P, int v, int sms, cudaStream_t s)
{
    switch (v) {
#define KERR_CASE(i, b, m, rm) \
    case i:                    \
        return launch_one<0, b, m, rm>(P, sms, s, true);
        KERR_VARIANT_LIST_HI(KERR_CASE)
#undef KERR_CASE
    default:
        return launch_trace_f32x2(P, v, sms, s);
    }
}

} // namespace kerr
