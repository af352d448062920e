// FP32+Kahan path: set-up, persistent stepping (FP32 phase and FP64-zone
// phase) and finishing launches.
#include "kerr_trace.cuh"
#include "kerr_variants.h"

namespace kerr {

static int grid_for(long long n, int block, int sms)
{
    long long g = (n + block - 1) / block;
    const long long cap = (long long)sms * 8;
    if (g > cap)
        g = cap;
    return g < 1 ? 1 : (int)g;
}

cudaError_t launch_setup_f32(const TraceParams &P, int sms, cudaStream_t s)
{
    f32_setup_kernel<<<grid_for(P.n, 256, sms), 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_finish_f32(const TraceParams &P, int sms, cudaStream_t s)
{
    f32_finish_kernel<<<grid_for(P.n, 256, sms), 256, 0, s>>>(P);
    return cudaGetLastError();
}

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

// Variants 0-4 are compiled here, 5-9 in kerr_trace_f32b.cu (in parallel).
cudaError_t launch_trace_f32_hi(const TraceParams &P, int v, int sms, cudaStream_t s);

cudaError_t launch_trace_f32(const TraceParams &P, int v, int sms, cudaStream_t s)
{
    switch (v) {
#define KERR_CASE(i, b, m, rm) \
    case i:                    \
        return launch_one<0, b, m, rm>(P, sms, s, true);
        KERR_VARIANT_LIST_LO(KERR_CASE)
#undef KERR_CASE
    default:
        return launch_trace_f32_hi(P, v, sms, s);
    }
}

} // namespace kerr
