// kerr_static.cu -- kerr_trace_camera_static: the camera entry point for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: real-time or embedded hosts that must
// not touch the allocator once they are running (cudaMalloc and cudaFree can
// synchronise the whole device and their latency is unbounded), and hosts
// whose device memory is owned and budgeted by another framework's pool, so
// that a library allocating behind their back breaks their accounting.  For
// them this entry point keeps
// every byte of its scratch -- work-queue and statistics counters, the camera
// table, the per-geodesic state and constant planes, the deferred-clip queue
// and the FP64-zone buffer -- in one file-scope device array of fixed size.  The caller still passes
// the output buffers, which must be device memory.
//
// The array is a static __device__ symbol, so every GPU that loads the library
// holds KERR_STATIC_SCRATCH_BYTES until the process exits, and every call
// shares it: it keeps the last call's contents, the counters are cleared at
// the start of each call, and calls that overlap on the GPU (other streams,
// other host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/kerr.h"
#define KERR_TYPES_ONLY
#include "kerr_trace.cuh"
#include "kerr_variants.h"

using namespace kerr;

namespace {

constexpr int64_t kMaxGeo = KERR_STATIC_MAX_GEODESICS;
constexpr int kMaxCams = KERR_STATIC_MAX_CAMERAS;
constexpr int64_t kZoneCap = kMaxGeo;      // one zone entry per geodesic
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Layout of the scratch array (byte offsets, each part 256-byte aligned).
constexpr size_t kCountersWords = kCounterWords(SC_COUNT);   // queue, stats, zone and clip counts
constexpr size_t kOffCounters = 0;
constexpr size_t kOffCams = align_up(kOffCounters + kCountersWords * sizeof(unsigned long long));
constexpr size_t kOffWork = align_up(kOffCams + kMaxCams * sizeof(CamDev));
constexpr size_t kOffZone = align_up(kOffWork + (size_t)kMaxGeo * kWorkBytesPerGeodesic);
constexpr size_t kBytes = align_up(kOffZone + (size_t)kZoneCap * sizeof(ZoneEntry));
static_assert(kBytes == KERR_STATIC_SCRATCH_BYTES, "kerr.h states the scratch size");

// In host code this name is only a host-side stand-in for the device array;
// kernels get the address returned by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_dev_ptr[kMaxDevices] = {};

int fail(int code, const char *msg) { return kerr_set_error(code, msg); }

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device address of the scratch array on the current device; looked up once
// per device (with that device current) and cached.
int scratch_ptr(int dev, char **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return fail(KERR_EINVAL, "kerr_trace_camera_static: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(KERR_ECUDA, "kerr_trace_camera_static: cudaGetSymbolAddress failed");
        }
        g_dev_ptr[dev] = p;
    }
    *out = (char *)g_dev_ptr[dev];
    return KERR_OK;
}

// The camera table travels to the device as a kernel argument (captured by
// value when the kernel is launched), so no host copy of it has to outlive
// the call and no pageable-memory copy is involved.
struct CamTable {
    CamDev c[kMaxCams];
};
static_assert(sizeof(CamTable) <= 4000, "kernel argument size");

__global__ void upload_cams_kernel(const CamTable t, int ncam, CamDev *dst)
{
    const int i = threadIdx.x;
    if (i < ncam)
        dst[i] = t.c[i];
}

} // namespace

extern "C" int kerr_trace_camera_static(const kerr_camera *cams, int32_t ncam,
                                        const kerr_opts *o, double *x_out, double *k_out,
                                        int32_t *status, int32_t *steps, float *diag,
                                        float *cross, void *stream)
{
    if (!cams || ncam < 1 || ncam > kMaxCams)
        return fail(KERR_EINVAL, "kerr_trace_camera_static: need 1..KERR_STATIC_MAX_CAMERAS cameras");
    // the same checks as kerr_trace_camera
    int rc = check_opts(o);
    if (rc)
        return rc;
    CamTable table;
    int64_t n = 0;
    rc = build_cams(cams, ncam, table.c, &n);
    if (rc)
        return rc;
    if (n > kMaxGeo)
        return fail(KERR_EINVAL, "kerr_trace_camera_static: more rays than "
                                 "KERR_STATIC_MAX_GEODESICS; use kerr_trace_camera");
    if (!is_device_ptr(x_out) || !is_device_ptr(k_out) || !is_device_ptr(status) ||
        !is_device_ptr(steps) || (diag && !is_device_ptr(diag)) ||
        (cross && !is_device_ptr(cross)))
        return fail(KERR_EINVAL, "kerr_trace_camera_static: outputs must be device memory "
                                 "(host buffers would need staging allocations)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ECUDA, "kerr_trace_camera_static: cudaGetDevice failed");
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ECUDA, "kerr_trace_camera_static: cudaDeviceGetAttribute failed");
    }
    char *base = nullptr;
    rc = scratch_ptr(dev, &base);
    if (rc)
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *ctr = (unsigned long long *)(base + kOffCounters);
    CamDev *dcams = (CamDev *)(base + kOffCams);
    char *work = base + kOffWork;
    ZoneEntry *zone = (ZoneEntry *)(base + kOffZone);

    // the previous call's counters are still in the array: clear them
    cudaError_t e = cudaMemsetAsync(ctr, 0, kCountersWords * sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        upload_cams_kernel<<<1, kMaxCams, 0, s>>>(table, ncam, dcams);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ECUDA, "kerr_trace_camera_static: clearing the scratch failed");
    }

    TraceParams P;
    std::memset(&P, 0, sizeof P);
    P.mode = MODE_CAMERA;
    P.n = n;
    P.cams = dcams;
    P.ncam = ncam;
    P.x_out = x_out;
    P.k_out = k_out;
    P.status = status;
    P.steps = steps;
    P.diag = diag;
    P.cross = cross;
    P.tol = o->tol;
    P.h0 = o->h0;
    P.max_steps = o->max_steps;
    P.r_escape = o->r_escape;
    P.t_end = o->t_end;
    P.fp64_zone = o->prec == KERR_FP32_KAHAN ? o->fp64_zone : 0.0;
    P.renorm_every = o->renorm_every;
    P.clip_maxit = o->clip_maxit;
    P.zone_df = o->zone_prec == KERR_ZONE_F32X2 ? 1 : 0;
    P.zone_quantum = o->zone_quantum;
    P.budget_ns = o->budget_ns;
    P.head = ctr;
    P.stats = ctr + 1;
    P.zcount = ctr + 1 + SC_COUNT;
    P.zhead = ctr + 2 + SC_COUNT;
    P.zpush = ctr + 3 + SC_COUNT;
    const int variant = o->variant >= 0 ? o->variant : kDefaultVariant[o->prec == KERR_FP32_KAHAN];
    if (o->prec == KERR_FP32_KAHAN) {
        bind_f32_scratch(P, work, ctr, n);
        if (P.fp64_zone > 0.0) {
            P.zbuf = zone;
            P.zcap = kZoneCap;
        }
        e = launch_setup_f32(P, sms, s);
        if (e == cudaSuccess)
            e = launch_trace_f32(P, variant, sms, s);
        if (e == cudaSuccess && P.zbuf)
            e = launch_zone_phase(P, o->zone_variant >= 0 ? o->zone_variant : kDefaultZoneVariant,
                                  sms, s);
        if (e == cudaSuccess)
            e = launch_clip_f32(P, sms, s);
        if (e == cudaSuccess)
            e = launch_finish_f32(P, sms, s);
    } else {
        e = launch_trace_f64(P, variant, sms, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ECUDA, "kerr_trace_camera_static: kernel launch failed");
    }
    return KERR_OK;
}
