// FP32 path, zone phase: continues the geodesics that the FP32 stepping
// phase deferred to the FP64 zone (its own translation unit so that it
// compiles in parallel with the stepping kernels).
#include "kerr_trace.cuh"
#include "kerr_variants.h"

namespace kerr {

// The FP64-zone phase: continues the geodesics deferred by the FP32 phase
// (float-float zone steps use one launch shape: their register demand leaves
// no room to choose).
// Its item count lives on the device, so the grid is fixed by the launch
// shape (blocks per SM x SMs); threads with nothing to do exit at once.
template <int PH, int B, int BPS, int RM, bool TEAM = false>
static cudaError_t launch_zone(const TraceParams &P, int sms, cudaStream_t s)
{
    trace_f32_kernel<PH, B, BPS, RM, TEAM><<<(unsigned)(BPS * sms), B, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_clip_f32(const TraceParams &P, int sms, cudaStream_t s)
{
    f32_clip_kernel<<<(unsigned)(4 * sms), 128, 0, s>>>(P);
    return cudaGetLastError();
}

void bind_f32_scratch(TraceParams &P, void *work, unsigned long long *ctr, int64_t n)
{
    static_assert(KC_COUNT == 9, "kWorkBytesPerGeodesic counts 9 constant planes");
    static_assert(kWorkBytesPerGeodesic == 120, "FP32-path scratch layout");
    char *w = static_cast<char *>(work);
    const size_t nn = (size_t)n;
    P.s_state = reinterpret_cast<float *>(w);
    P.s_const = P.s_state + 16 * nn;
    P.clip_h = P.s_const + (size_t)KC_COUNT * nn;
    P.clip_shi = reinterpret_cast<double *>(w + (16 + KC_COUNT + 1) * sizeof(float) * nn);
    P.clipq = reinterpret_cast<int64_t *>(P.clip_shi + nn);
    P.head = ctr;
    P.stats = ctr + 1;
    P.zcount = ctr + 1 + SC_COUNT;
    P.zhead = ctr + 2 + SC_COUNT;
    P.zpush = ctr + 3 + SC_COUNT;
    P.cq32 = ctr + 4 + SC_COUNT;
    P.cq64 = ctr + 5 + SC_COUNT;
    P.zdone = ctr + 6 + SC_COUNT;
}

cudaError_t launch_zone_phase(const TraceParams &P, int zv, int sms, cudaStream_t s)
{
    switch (zv) {
#define KERR_ZCASE(i, b, m, rm)                                                        \
    case i:                                                                            \
        return P.zone_df ? launch_zone<2, 128, 2, RHS_CALL>(P, sms, s)                   \
                         : launch_zone<1, b, m, rm>(P, sms, s);
        KERR_ZONE_VARIANT_LIST(KERR_ZCASE)
#undef KERR_ZCASE
    case kTeamZoneVariant:
        return P.zone_df ? launch_zone<2, 128, 2, RHS_CALL>(P, sms, s)
                         : launch_zone<1, 128, 1, RHS_CALL, true>(P, sms, s);
    case kTeamPairZoneVariant:
        return P.zone_df ? launch_zone<2, 128, 2, RHS_CALL>(P, sms, s)
                         : launch_zone<1, 128, 1, RHS_PAIR, true>(P, sms, s);
    default:
        return cudaErrorInvalidValue;
    }
}

} // namespace kerr
