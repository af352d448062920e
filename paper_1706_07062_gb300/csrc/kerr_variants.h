// kerr_variants.h -- launch configurations of the persistent kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kerr.h"

namespace kerr {

// (threads per block, minimum resident blocks per SM).  The second number
// caps registers per thread at 65536 / (block * min_blocks).
struct Variant {
    int block, min_blocks;
};

// Stepping-kernel variants: (index, threads per block, minimum blocks per SM,
// FP32-phase right-hand sides: 0 inline, 1 one out-of-line copy).  The FP64
// path uses the launch shape only (its right-hand sides are out of line).
#define KERR_VARIANT_LIST_LO(X) X(0, 128, 4, 0) X(1, 128, 3, 0) X(2, 256, 2, 0) X(3, 128, 4, 1) \
    X(4, 128, 3, 1)
#define KERR_VARIANT_LIST_HI(X) X(5, 128, 2, 0) X(6, 64, 8, 0) X(7, 128, 5, 0) X(8, 256, 2, 1) \
    X(9, 128, 5, 1)
#define KERR_VARIANT_LIST(X) KERR_VARIANT_LIST_LO(X) KERR_VARIANT_LIST_HI(X)
// FP32 stepping with two geodesics per thread (packed f32x2 right-hand sides,
// always out of line): (index, threads per block, minimum blocks per SM).
// FP32+Kahan path only.
#define KERR_VARIANT_LIST_X2(X) X(10, 128, 2) X(11, 128, 3) X(12, 64, 4) X(13, 64, 6)

constexpr int kNumVariants = 14;
constexpr int kFirstX2Variant = 10;
// Defaults before autotuning, per precision (KERR_FP64, KERR_FP32_KAHAN):
// the fastest on the 1024 x 1024, a = 0.99 camera.
constexpr int kDefaultVariant[2] = {1, 8};
constexpr Variant kVariants[kNumVariants] = {{128, 4}, {128, 3}, {256, 2}, {128, 4}, {128, 3},
                                             {128, 2}, {64, 8},  {128, 5}, {256, 2}, {128, 5},
                                             {128, 2}, {128, 3}, {64, 4},  {64, 6}};
// Geodesics per thread of each variant.
constexpr int kVariantRays[kNumVariants] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2};
// Right-hand-side mode of each variant's FP32 steps (RHS_INLINE = 0, RHS_CALL = 1).
constexpr int kVariantRhs[kNumVariants] = {0, 0, 0, 1, 1, 0, 0, 0, 1, 1, 1, 1, 1, 1};

// Zone-phase variants: (threads per block, blocks per SM, how FP64 steps
// evaluate their right-hand sides: 0 inline, 1 one out-of-line copy, 2
// out-of-line pairs -- see RHS_INLINE / RHS_CALL / RHS_PAIR).  Variants 7 and
// 8 are variants 3 and 4 with two-lane zone attempts in the phase's tail
// (TEAM).
#define KERR_ZONE_VARIANT_LIST(X)                                                          \
    X(0, 128, 2, 0) X(1, 128, 1, 0) X(2, 64, 2, 0) X(3, 128, 1, 1) X(4, 128, 1, 2)          \
    X(5, 128, 2, 2) X(6, 64, 2, 2)
constexpr int kNumZoneVariants = 9;
constexpr int kTeamZoneVariant = 7;
constexpr int kTeamPairZoneVariant = 8;
constexpr Variant kZoneVariants[kNumZoneVariants] = {{128, 2}, {128, 1}, {64, 2},
                                                     {128, 1}, {128, 1}, {128, 2},
                                                     {64, 2},  {128, 1}, {128, 1}};
constexpr int kDefaultZoneVariant = kTeamZoneVariant;

struct TraceParams;

// Launch the persistent kernel for variant v on a grid of `blocks_per_sm *
// sms` blocks (0 = as many as fit).  Returns the CUDA error of the launch.
cudaError_t launch_trace_f32(const TraceParams &P, int v, int sms, cudaStream_t s);
cudaError_t launch_trace_f32x2(const TraceParams &P, int v, int sms, cudaStream_t s);
cudaError_t launch_trace_f64(const TraceParams &P, int v, int sms, cudaStream_t s);
cudaError_t launch_zone_phase(const TraceParams &P, int zv, int sms, cudaStream_t s);
cudaError_t launch_setup_f32(const TraceParams &P, int sms, cudaStream_t s);
cudaError_t launch_finish_f32(const TraceParams &P, int sms, cudaStream_t s);
// Clip pass of the FP32 path (geodesics whose clipping was deferred).
cudaError_t launch_clip_f32(const TraceParams &P, int sms, cudaStream_t s);

// FP32-path scratch per geodesic: state and constant planes, then the
// deferred-clip step length (float), event value (double) and queue (int64).
constexpr size_t kWorkBytesPerGeodesic = (16 + 9) * sizeof(float) + sizeof(float) +
                                         sizeof(double) + sizeof(int64_t);
// Counters ahead of the FP32 path's scratch: queue head, statistics, zone
// count / head / re-queue count, clip-queue counts (FP32 front, zone back),
// zone geodesics finished.
constexpr int kCounterWords(int sc_count) { return 1 + sc_count + 3 + 2 + 1; }

// Points the FP32 path's scratch pointers of P into `work` (n geodesics,
// kWorkBytesPerGeodesic each, 8-byte aligned) and `ctr` (kCounterWords).
void bind_f32_scratch(TraceParams &P, void *work, unsigned long long *ctr, int64_t n);

struct CoordParams;
// Coordinate-time integration in FP64 (fp32 = 0) or FP32 with compensated
// state updates (fp32 = 1), persistent grid over `sms` SMs.
cudaError_t launch_coordtime(const CoordParams &P, int fp32, int sms, cudaStream_t s);

// Resident blocks per SM (at least 1) of kernel `fn` launched with `block`
// threads and no dynamic shared memory on the current device.  Looked up once
// per (kernel, device) and cached under a lock, so that a process that drives
// several GPUs, or calls from several host threads, gets each device's value.
cudaError_t blocks_per_sm(const void *fn, int block, int *out);

// Checks shared by the trace entry points (KERR_OK, or the error code with
// kerr_last_error() set): the options, and a camera list, which is converted
// to the kernels' table out[0 .. ncam-1] with *n = the total number of rays.
int check_opts(const kerr_opts *o);
struct CamDev;
int build_cams(const kerr_camera *cams, int32_t ncam, CamDev *out, int64_t *n);

// Device allocation used by every library-owned buffer: cudaMalloc, unless
// an injected failure is armed (kerr_debug_fail_alloc), in which case the
// chosen allocation reports cudaErrorMemoryAllocation without allocating.
cudaError_t dev_alloc_bytes(void **p, size_t bytes);
template <typename T> inline cudaError_t dev_alloc(T **p, size_t bytes)
{
    return dev_alloc_bytes(reinterpret_cast<void **>(p), bytes);
}

// Records `msg` as this thread's kerr_last_error() and returns `code`.
int kerr_set_error(int code, const char *msg);

} // namespace kerr
