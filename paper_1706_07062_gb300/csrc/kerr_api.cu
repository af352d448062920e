// kerr_api.cu -- the C ABI declared in include/kerr.h: argument checks,
// host/device staging, the work-queue and statistics scratch, CUDA-graph
// replay of the integration launch, and the launch-configuration autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/kerr.h"
#define KERR_TYPES_ONLY
#include "kerr_trace.cuh"
#include "kerr_variants.h"

using namespace kerr;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define KERR_CUDA(call)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(KERR_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));           \
    } while (0)

bool is_device_ptr(const void *p)
{
    if (!p)
        return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The device's address of page-locked host memory (cudaHostAlloc,
// cudaHostRegister), or null for any other pointer.
void *mapped_host_ptr(void *p)
{
    if (!p)
        return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

} // namespace

// Launch parameters that identify a cached graph.
struct GraphKey {
    TraceParams P;
    int variant;
    int zone_variant;
    int f32;
    bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof *this) == 0; }
};

struct kerr_ctx {
    double a = 0.0;
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;               // the context's own stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_k0 = nullptr, ev_k1 = nullptr;
    cudaEvent_t ev_ph[3] = {nullptr, nullptr, nullptr};   // phase boundaries (in the graph)
    unsigned long long *d_scratch = nullptr;     // [0] queue head, [1..16] statistics,
                                                 // [17] zone count, [18] zone-phase head
    ZoneEntry *d_zone = nullptr;                 // deferred FP64-zone geodesics
    int64_t zone_cap = 0;
    char *d_work = nullptr;                      // FP32 path: state, constants, clip queue
    int64_t work_cap = 0;                        // geodesics d_work can hold
    CamDev *d_cams = nullptr;
    int cam_cap = 0;
    char *d_stage = nullptr;                     // staging arena for host buffers
    size_t stage_cap = 0;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;
    bool gvalid = false;
    int32_t *h_abort = nullptr;                  // abort flag: mapped pinned host memory
    int32_t *d_abort = nullptr;                  // ... and its device address
    int tuned[2] = {-1, -1};                     // autotuned variant per precision
    int tuned_zone[2] = {-1, -1};                // autotuned zone-phase variant per precision
    int last_variant = -1;
    int last_f32 = 0;
    bool have_stats = false;
};

static const int kScratchWords = kCounterWords(SC_COUNT);

extern "C" void kerr_opts_default(kerr_opts *o)
{
    if (!o)
        return;
    std::memset(o, 0, sizeof *o);
    o->prec = KERR_FP32_KAHAN;
    o->renorm_every = 0;
    o->tol = 1e-6;
    o->h0 = 1.0;
    o->max_steps = 1000000;
    o->r_escape = 0.0;
    o->t_end = INFINITY;
    o->fp64_zone = 1.5;
    o->clip_maxit = 40;
    o->variant = -1;
    o->budget_ns = 0;
    o->zone_prec = KERR_ZONE_FP64;
    o->zone_variant = -1;
    o->zone_quantum = 32;
}

extern "C" const char *kerr_last_error(void) { return g_err.c_str(); }

int kerr::kerr_set_error(int code, const char *msg)
{
    g_err = msg;
    return code;
}

// Injected allocation failure: the n-th next library allocation fails.
static std::atomic<int> g_fail_alloc{0};

cudaError_t kerr::dev_alloc_bytes(void **p, size_t bytes)
{
    int n = g_fail_alloc.load();
    while (n > 0) {
        if (g_fail_alloc.compare_exchange_weak(n, n - 1)) {
            if (n == 1) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

extern "C" int kerr_debug_fail_alloc(int32_t n)
{
    if (n < 0)
        return fail(KERR_EINVAL, "kerr_debug_fail_alloc: n = %d < 0", n);
    g_fail_alloc.store(n);
    return KERR_OK;
}

cudaError_t kerr::blocks_per_sm(const void *fn, int block, int *out)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;   // (kernel, device) -> blocks
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    const auto key = std::make_pair(fn, dev * 4096 + block);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it == cache.end()) {
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, 0);
        if (e != cudaSuccess)
            return e;
        it = cache.emplace(key, n < 1 ? 1 : n).first;
    }
    *out = it->second;
    return cudaSuccess;
}

extern "C" int kerr_num_variants(void) { return kNumVariants; }

extern "C" int kerr_variant_info(int v, int32_t *block, int32_t *min_blocks)
{
    if (v < 0 || v >= kNumVariants)
        return fail(KERR_EINVAL, "variant %d out of range [0, %d)", v, kNumVariants);
    if (block)
        *block = kVariants[v].block;
    if (min_blocks)
        *min_blocks = kVariants[v].min_blocks;
    return KERR_OK;
}

extern "C" int kerr_variant_shape(int v, int32_t *block, int32_t *min_blocks,
                                  int32_t *rays_per_thread, int32_t *rhs_mode)
{
    if (v < 0 || v >= kNumVariants)
        return fail(KERR_EINVAL, "variant %d out of range [0, %d)", v, kNumVariants);
    if (block)
        *block = kVariants[v].block;
    if (min_blocks)
        *min_blocks = kVariants[v].min_blocks;
    if (rays_per_thread)
        *rays_per_thread = kVariantRays[v];
    if (rhs_mode)
        *rhs_mode = kVariantRhs[v];
    return KERR_OK;
}

extern "C" int kerr_num_zone_variants(void) { return kNumZoneVariants; }

extern "C" int kerr_zone_variant_info(int v, int32_t *block, int32_t *blocks_per_sm)
{
    if (v < 0 || v >= kNumZoneVariants)
        return fail(KERR_EINVAL, "zone variant %d out of range [0, %d)", v, kNumZoneVariants);
    if (block)
        *block = kZoneVariants[v].block;
    if (blocks_per_sm)
        *blocks_per_sm = kZoneVariants[v].min_blocks;
    return KERR_OK;
}

extern "C" int kerr_init(double a, kerr_ctx **out)
{
    if (!out)
        return fail(KERR_EINVAL, "kerr_init: out is NULL");
    *out = nullptr;
    if (!(std::fabs(a) <= 1.0))
        return fail(KERR_EINVAL, "kerr_init: spin a = %g outside [-1, 1]", a);
    kerr_ctx *c = new (std::nothrow) kerr_ctx();
    if (!c)
        return fail(KERR_ENOMEM, "kerr_init: out of host memory");
    c->a = a;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreate(&c->ev_k0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&c->ev_k1);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        e = cudaEventCreate(&c->ev_ph[i]);
    if (e == cudaSuccess)
        e = dev_alloc(&c->d_scratch, kScratchWords * sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = cudaMemset(c->d_scratch, 0, kScratchWords * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        int code = (e == cudaErrorMemoryAllocation) ? KERR_ENOMEM : KERR_ECUDA;
        kerr_destroy(c);
        return fail(code, "kerr_init: %s", cudaGetErrorString(e));
    }
    *out = c;
    return KERR_OK;
}

extern "C" int kerr_destroy(kerr_ctx *c)
{
    if (!c)
        return KERR_OK;
    if (c->stream)
        cudaStreamSynchronize(c->stream);
    if (c->gexec)
        cudaGraphExecDestroy(c->gexec);
    cudaFree(c->d_scratch);
    cudaFree(c->d_zone);
    cudaFree(c->d_work);
    cudaFree(c->d_cams);
    cudaFree(c->d_stage);
    if (c->h_abort)
        cudaFreeHost(c->h_abort);
    if (c->ev_in)
        cudaEventDestroy(c->ev_in);
    if (c->ev_out)
        cudaEventDestroy(c->ev_out);
    if (c->ev_k0)
        cudaEventDestroy(c->ev_k0);
    if (c->ev_k1)
        cudaEventDestroy(c->ev_k1);
    for (int i = 0; i < 3; ++i)
        if (c->ev_ph[i])
            cudaEventDestroy(c->ev_ph[i]);
    if (c->stream)
        cudaStreamDestroy(c->stream);
    delete c;
    return KERR_OK;
}

int kerr::check_opts(const kerr_opts *o)
{
    if (!o)
        return fail(KERR_EINVAL, "opts is NULL");
    if (o->prec != KERR_FP64 && o->prec != KERR_FP32_KAHAN)
        return fail(KERR_EINVAL, "opts.prec = %d is not KERR_FP64 or KERR_FP32_KAHAN", o->prec);
    if (!(o->tol > 0.0) || !std::isfinite(o->tol))
        return fail(KERR_EINVAL, "opts.tol = %g must be finite and > 0", o->tol);
    if (!(o->h0 > 0.0) || !std::isfinite(o->h0))
        return fail(KERR_EINVAL, "opts.h0 = %g must be finite and > 0", o->h0);
    if (o->max_steps < 0)
        return fail(KERR_EINVAL, "opts.max_steps = %lld < 0", (long long)o->max_steps);
    if (std::isnan(o->r_escape))
        return fail(KERR_EINVAL, "opts.r_escape is NaN");
    if (!(o->fp64_zone >= 0.0))
        return fail(KERR_EINVAL, "opts.fp64_zone = %g < 0", o->fp64_zone);
    if (o->clip_maxit < 1)
        return fail(KERR_EINVAL, "opts.clip_maxit = %d < 1", o->clip_maxit);
    if (o->renorm_every < 0)
        return fail(KERR_EINVAL, "opts.renorm_every = %d < 0", o->renorm_every);
    if (o->zone_prec != KERR_ZONE_FP64 && o->zone_prec != KERR_ZONE_F32X2)
        return fail(KERR_EINVAL, "opts.zone_prec = %d is not KERR_ZONE_FP64 or KERR_ZONE_F32X2",
                    o->zone_prec);
    if (o->variant < -1 || o->variant >= kNumVariants)
        return fail(KERR_EINVAL, "opts.variant = %d outside [-1, %d)", o->variant, kNumVariants);
    if (o->prec == KERR_FP64 && o->variant >= 0 && kVariantRays[o->variant] != 1)
        return fail(KERR_EINVAL, "opts.variant = %d (two geodesics per thread) is FP32-only",
                    o->variant);
    if (o->zone_quantum < 0)
        return fail(KERR_EINVAL, "opts.zone_quantum = %d < 0", o->zone_quantum);
    if (o->zone_variant < -1 || o->zone_variant >= kNumZoneVariants)
        return fail(KERR_EINVAL, "opts.zone_variant = %d outside [-1, %d)", o->zone_variant,
                    kNumZoneVariants);
    return KERR_OK;
}

// Staging of host buffers through a library-owned device arena.
struct Stage {
    const void *host;
    void **dev;     // where to put the device pointer
    size_t bytes;
    bool input;
    size_t off;
};

static int ensure_stage(kerr_ctx *c, size_t bytes)
{
    if (bytes <= c->stage_cap)
        return KERR_OK;
    cudaStreamSynchronize(c->stream);
    cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_cap = 0;
    size_t cap = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = dev_alloc(&c->d_stage, cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ENOMEM, "staging allocation of %zu bytes failed: %s", cap,
                    cudaGetErrorString(e));
    }
    c->stage_cap = cap;
    return KERR_OK;
}

static int launch_integration(kerr_ctx *c, const TraceParams &P, int prec, int variant,
                              int zone_variant)
{
    const int f32 = (prec == KERR_FP32_KAHAN) ? 1 : 0;
    GraphKey key;
    std::memset(&key, 0, sizeof key);
    key.P = P;
    key.variant = variant;
    key.zone_variant = zone_variant;
    key.f32 = f32;
    if (!(c->gvalid && c->gkey == key)) {
        cudaGraph_t g = nullptr;
        KERR_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = cudaMemsetAsync(c->d_scratch, 0, kScratchWords * sizeof(unsigned long long),
                                         c->stream);
        cudaError_t e2 = e1;
        // event-record nodes (external records, so that they can be timed)
        // between the launches time each phase
        if (f32) {
            if (e2 == cudaSuccess)
                e2 = launch_setup_f32(P, c->sms, c->stream);
            if (e2 == cudaSuccess)
                e2 = cudaEventRecordWithFlags(c->ev_ph[0], c->stream, cudaEventRecordExternal);
            if (e2 == cudaSuccess)
                e2 = launch_trace_f32(P, variant, c->sms, c->stream);
            if (e2 == cudaSuccess)
                e2 = cudaEventRecordWithFlags(c->ev_ph[1], c->stream, cudaEventRecordExternal);
            if (e2 == cudaSuccess && P.zbuf)
                e2 = launch_zone_phase(P, zone_variant, c->sms, c->stream);
            if (e2 == cudaSuccess)
                e2 = cudaEventRecordWithFlags(c->ev_ph[2], c->stream, cudaEventRecordExternal);
            if (e2 == cudaSuccess && P.clipq)
                e2 = launch_clip_f32(P, c->sms, c->stream);
            if (e2 == cudaSuccess)
                e2 = launch_finish_f32(P, c->sms, c->stream);
        } else if (e2 == cudaSuccess) {
            e2 = launch_trace_f64(P, variant, c->sms, c->stream);
        }
        cudaError_t e3 = cudaStreamEndCapture(c->stream, &g);
        if (e2 != cudaSuccess || e3 != cudaSuccess) {
            if (g)
                cudaGraphDestroy(g);
            cudaGetLastError();
            return fail(KERR_ECUDA, "graph capture failed: %s",
                        cudaGetErrorString(e2 != cudaSuccess ? e2 : e3));
        }
        bool updated = false;
        if (c->gexec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(c->gexec, g, &info) == cudaSuccess)
                updated = true;
            else {
                cudaGetLastError();
                cudaGraphExecDestroy(c->gexec);
                c->gexec = nullptr;
            }
        }
        if (!updated) {
            cudaError_t e = cudaGraphInstantiate(&c->gexec, g, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(g);
                c->gvalid = false;
                return fail(KERR_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
            }
        }
        cudaGraphDestroy(g);
        c->gkey = key;
        c->gvalid = true;
    }
    KERR_CUDA(cudaEventRecord(c->ev_k0, c->stream));
    KERR_CUDA(cudaGraphLaunch(c->gexec, c->stream));
    KERR_CUDA(cudaEventRecord(c->ev_k1, c->stream));
    c->last_variant = variant;
    c->last_f32 = f32;
    c->have_stats = true;
    return KERR_OK;
}

// Shared body of the three trace entry points.
// Extra launch inputs of the internal callers (surrogate fallback).
struct TraceExtra {
    const double *points = nullptr;
    double r_obs = 0.0;
    const int64_t *index = nullptr;                 // device
    const unsigned long long *n_dev = nullptr;      // device
    double *traj = nullptr;                         // device, FP64 path: stored solution
    int32_t traj_cap = 0;
    int32_t *traj_count = nullptr;                  // device
};

static int trace_common(kerr_ctx *c, int mode, const double *x0, const double *k0,
                        const double *t_end_each, int64_t n,
                        const CamDev *cams_host, int32_t ncam, const kerr_opts *o, double *x_out,
                        double *k_out, int32_t *status, int32_t *steps, float *diag, float *cross,
                        void *stream, const TraceExtra &X = TraceExtra())
{
    if (!c)
        return fail(KERR_EINVAL, "context is NULL");
    int rc = check_opts(o);
    if (rc)
        return rc;
    if (n < 0)
        return fail(KERR_EINVAL, "n = %lld < 0", (long long)n);
    if (n == 0)
        return KERR_OK;
    if (!x_out || !k_out || !status || !steps)
        return fail(KERR_EINVAL, "x_out, k_out, status and steps must not be NULL");
    if ((mode == MODE_RAYS || mode == MODE_PARTICLES) && (!x0 || !k0))
        return fail(KERR_EINVAL, "input planes must not be NULL");
    if (mode == MODE_POINTS && !X.points)
        return fail(KERR_EINVAL, "points must not be NULL");
    cudaStream_t us = (cudaStream_t)stream;

    TraceParams P;
    std::memset(&P, 0, sizeof P);
    P.mode = mode;
    P.n = n;
    P.a = c->a;
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
    P.abort = c->d_abort;
    P.head = c->d_scratch;
    P.stats = c->d_scratch + 1;
    P.zcount = c->d_scratch + 1 + SC_COUNT;
    P.zhead = c->d_scratch + 2 + SC_COUNT;
    P.zpush = c->d_scratch + 3 + SC_COUNT;
    if (o->prec == KERR_FP32_KAHAN) {
        // state [16][n] and constant [KC_COUNT][n] float planes, deferred-clip
        // planes and queue
        if (n > c->work_cap) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->d_work);
            c->d_work = nullptr;
            c->work_cap = 0;
            cudaError_t e = dev_alloc(&c->d_work, (size_t)n * kWorkBytesPerGeodesic);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(KERR_ENOMEM, "work buffer allocation (%lld geodesics) failed",
                            (long long)n);
            }
            c->work_cap = n;
        }
        bind_f32_scratch(P, c->d_work, c->d_scratch, n);
    }
    if (o->prec == KERR_FP32_KAHAN && o->fp64_zone > 0.0) {
        // Deferred-zone buffer: one entry per geodesic (each is deferred at
        // most once), so the stepping phase never steps in the zone itself --
        // an in-place FP64 step in that kernel cost it registers and spills.
        const int64_t want = n;
        if (want > c->zone_cap) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->d_zone);
            c->d_zone = nullptr;
            c->zone_cap = 0;
            cudaError_t e = dev_alloc(&c->d_zone, (size_t)want * sizeof(ZoneEntry));
            if (e == cudaSuccess)    // queue slots start empty (seq = 0)
                e = cudaMemset(c->d_zone, 0, (size_t)want * sizeof(ZoneEntry));
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(KERR_ENOMEM, "zone buffer allocation (%lld entries) failed",
                            (long long)want);
            }
            c->zone_cap = want;
        }
        P.zbuf = c->d_zone;
        P.zcap = c->zone_cap;
    }

    // ---- which buffers live on the host
    const size_t nn = (size_t)n;
    const size_t in_planes = (mode == MODE_PARTICLES) ? 3 : 4;
    std::vector<Stage> st;
    P.x0 = x0;
    P.k0 = k0;
    P.t_end_each = t_end_each;
    P.x_out = x_out;
    P.k_out = k_out;
    P.status = status;
    P.steps = steps;
    P.diag = diag;
    P.cross = cross;
    P.points = X.points;
    P.r_obs = X.r_obs;
    P.index = X.index;
    P.n_dev = X.n_dev;
    P.traj = X.traj;
    P.traj_cap = X.traj_cap;
    P.traj_count = X.traj_count;
    if (mode == MODE_POINTS && !is_device_ptr(X.points))
        st.push_back({X.points, (void **)&P.points, 4 * nn * sizeof(double), true, 0});
    if (mode == MODE_RAYS || mode == MODE_PARTICLES) {
        if (!is_device_ptr(x0))
            st.push_back({x0, (void **)&P.x0, 4 * nn * sizeof(double), true, 0});
        if (!is_device_ptr(k0))
            st.push_back({k0, (void **)&P.k0, in_planes * nn * sizeof(double), true, 0});
        if (t_end_each && !is_device_ptr(t_end_each))
            st.push_back({t_end_each, (void **)&P.t_end_each, nn * sizeof(double), true, 0});
    }
    // End points and diagnostics are only written, once per geodesic, by the
    // kernels (the finishing pass of the FP32 path, the stepping kernel of the
    // FP64 path): page-locked host buffers receive them in place over the
    // host link, with no staging copy after the kernels; pageable ones are
    // staged.  Status, steps and crossings are also read by the kernels and
    // stay in device memory.
    bool written_in_place = false;
    if (!is_device_ptr(x_out)) {
        if (void *m = mapped_host_ptr(x_out)) {
            P.x_out = static_cast<double *>(m);
            written_in_place = true;
        } else {
            st.push_back({x_out, (void **)&P.x_out, 4 * nn * sizeof(double), false, 0});
        }
    }
    if (!is_device_ptr(k_out)) {
        if (void *m = mapped_host_ptr(k_out)) {
            P.k_out = static_cast<double *>(m);
            written_in_place = true;
        } else {
            st.push_back({k_out, (void **)&P.k_out, 4 * nn * sizeof(double), false, 0});
        }
    }
    if (!is_device_ptr(status))
        st.push_back({status, (void **)&P.status, nn * sizeof(int32_t), false, 0});
    if (!is_device_ptr(steps))
        st.push_back({steps, (void **)&P.steps, nn * sizeof(int32_t), false, 0});
    if (diag && !is_device_ptr(diag)) {
        if (void *m = mapped_host_ptr(diag)) {
            P.diag = static_cast<float *>(m);
            written_in_place = true;
        } else {
            st.push_back({diag, (void **)&P.diag, 4 * nn * sizeof(float), false, 0});
        }
    }
    if (cross && !is_device_ptr(cross))
        st.push_back({cross, (void **)&P.cross, 5 * nn * sizeof(float), false, 0});
    size_t total = 0;
    for (auto &s : st) {
        s.off = total;
        total += (s.bytes + 255) & ~(size_t)255;
    }
    if (total) {
        rc = ensure_stage(c, total);
        if (rc)
            return rc;
        for (auto &s : st)
            *s.dev = c->d_stage + s.off;
    }

    // ---- order after the caller's stream
    KERR_CUDA(cudaEventRecord(c->ev_in, us));
    KERR_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in, 0));

    if (mode == MODE_CAMERA) {
        if (ncam > c->cam_cap) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->d_cams);
            c->d_cams = nullptr;
            c->cam_cap = 0;
            cudaError_t e = dev_alloc(&c->d_cams, (size_t)ncam * sizeof(CamDev));
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(KERR_ENOMEM, "camera table allocation failed");
            }
            c->cam_cap = ncam;
        }
        // The camera table is small; copy it synchronously from a stack copy
        // so the caller's array can go out of scope.
        KERR_CUDA(cudaMemcpyAsync(c->d_cams, cams_host, (size_t)ncam * sizeof(CamDev),
                                  cudaMemcpyHostToDevice, c->stream));
        KERR_CUDA(cudaStreamSynchronize(c->stream));
        P.cams = c->d_cams;
        P.ncam = ncam;
    }
    for (auto &s : st)
        if (s.input)
            KERR_CUDA(cudaMemcpyAsync(*s.dev, s.host, s.bytes, cudaMemcpyHostToDevice, c->stream));

    int prec = o->prec;
    int variant = o->variant >= 0 ? o->variant
                                   : (c->tuned[prec] >= 0 ? c->tuned[prec] : kDefaultVariant[prec]);
    const int zvar = o->zone_variant >= 0
                         ? o->zone_variant
                         : (c->tuned_zone[prec] >= 0 ? c->tuned_zone[prec] : kDefaultZoneVariant);
    rc = launch_integration(c, P, prec, variant, zvar);
    if (rc)
        return rc;

    bool any_host = false;
    for (auto &s : st)
        if (!s.input) {
            KERR_CUDA(cudaMemcpyAsync((void *)s.host, *s.dev, s.bytes, cudaMemcpyDeviceToHost,
                                      c->stream));
            any_host = true;
        }
    for (auto &s : st)
        any_host = any_host || s.input;
    any_host = any_host || written_in_place;
    KERR_CUDA(cudaEventRecord(c->ev_out, c->stream));
    KERR_CUDA(cudaStreamWaitEvent(us, c->ev_out, 0));
    if (any_host)
        KERR_CUDA(cudaStreamSynchronize(c->stream));
    return KERR_OK;
}

extern "C" int kerr_abort_flag(kerr_ctx *c, int32_t **flag)
{
    if (!c || !flag)
        return fail(KERR_EINVAL, "kerr_abort_flag: NULL argument");
    if (!c->h_abort) {
        void *h = nullptr;
        cudaError_t e = cudaHostAlloc(&h, sizeof(int32_t), cudaHostAllocMapped);
        void *d = nullptr;
        if (e == cudaSuccess) {
            *(volatile int32_t *)h = 0;
            e = cudaHostGetDevicePointer(&d, h, 0);
        }
        if (e != cudaSuccess) {
            if (h)
                cudaFreeHost(h);
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? KERR_ENOMEM : KERR_ECUDA,
                        "kerr_abort_flag: mapped host allocation failed: %s",
                        cudaGetErrorString(e));
        }
        c->h_abort = (int32_t *)h;
        c->d_abort = (int32_t *)d;
    }
    *flag = c->h_abort;
    return KERR_OK;
}

extern "C" int kerr_trace_rays(kerr_ctx *c, const double *x0, const double *k0, int64_t n,
                               const kerr_opts *o, double *x_out, double *k_out, int32_t *status,
                               int32_t *steps, float *diag, float *cross, void *stream)
{
    return trace_common(c, MODE_RAYS, x0, k0, nullptr, n, nullptr, 0, o, x_out, k_out, status,
                        steps, diag, cross, stream);
}

extern "C" int kerr_trace_rays_dense(kerr_ctx *c, const double *x0, const double *k0, int64_t n,
                                     const kerr_opts *o, int32_t cap, double *traj,
                                     int32_t *traj_count, double *x_out, double *k_out,
                                     int32_t *status, int32_t *steps, void *stream)
{
    if (!o || o->prec != KERR_FP64)
        return fail(KERR_EINVAL, "kerr_trace_rays_dense: the stored solution needs the FP64 path");
    if (cap < 1)
        return fail(KERR_EINVAL, "kerr_trace_rays_dense: cap = %d < 1", cap);
    if (n > 0 && (!traj || !traj_count))
        return fail(KERR_EINVAL, "kerr_trace_rays_dense: NULL stored-solution buffer");
    if (n > 0 && (!is_device_ptr(traj) || !is_device_ptr(traj_count)))
        return fail(KERR_EINVAL, "kerr_trace_rays_dense: stored-solution buffers must be device memory");
    TraceExtra X;
    X.traj = traj;
    X.traj_cap = cap;
    X.traj_count = traj_count;
    return trace_common(c, MODE_RAYS, x0, k0, nullptr, n, nullptr, 0, o, x_out, k_out, status,
                        steps, nullptr, nullptr, stream, X);
}

extern "C" int kerr_trace_particles(kerr_ctx *c, const double *x0, const double *v0,
                                    const double *t_end, int64_t n, const kerr_opts *o,
                                    double *x_out, double *k_out, int32_t *status, int32_t *steps,
                                    float *diag, float *cross, void *stream)
{
    return trace_common(c, MODE_PARTICLES, x0, v0, t_end, n, nullptr, 0, o, x_out, k_out, status,
                        steps, diag, cross, stream);
}

static bool on_device(const void *p)
{
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
}

extern "C" int kerr_trace_coordtime(kerr_ctx *c, const double *x0, const double *v0,
                                    const double *t_end, int64_t n, const kerr_opts *o,
                                    double *x_out, double *v_out, int32_t *status,
                                    int32_t *steps, void *stream)
{
    if (!c)
        return fail(KERR_EINVAL, "kerr_trace_coordtime: NULL context");
    int rc = check_opts(o);
    if (rc)
        return rc;
    if (n < 0)
        return fail(KERR_EINVAL, "kerr_trace_coordtime: n = %lld < 0", (long long)n);
    if (n == 0)
        return KERR_OK;
    if (!x0 || !v0 || !x_out || !v_out || !status || !steps)
        return fail(KERR_EINVAL, "kerr_trace_coordtime: NULL buffer");
    if (!on_device(x0) || !on_device(v0) || !on_device(x_out) || !on_device(v_out) ||
        !on_device(status) || !on_device(steps) || (t_end && !on_device(t_end)))
        return fail(KERR_EINVAL, "kerr_trace_coordtime: buffers must be device memory");
    if (!t_end && std::isnan(o->t_end))
        return fail(KERR_EINVAL, "kerr_trace_coordtime: no end time (t_end NULL, opts.t_end NaN)");
    CoordParams P;
    std::memset(&P, 0, sizeof P);
    P.n = n;
    P.a = c->a;
    P.x0 = x0;
    P.v0 = v0;
    P.t_end_each = t_end;
    P.t_end = o->t_end;
    P.x_out = x_out;
    P.v_out = v_out;
    P.status = status;
    P.steps = steps;
    P.tol = o->tol;
    P.h0 = o->h0;
    P.r_escape = o->r_escape;
    P.max_steps = o->max_steps;
    P.head = c->d_scratch;
    P.stats = c->d_scratch + 1;
    cudaStream_t us = (cudaStream_t)stream;
    KERR_CUDA(cudaEventRecord(c->ev_in, us));
    KERR_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
    KERR_CUDA(cudaMemsetAsync(c->d_scratch, 0, kScratchWords * sizeof(unsigned long long),
                              c->stream));
    KERR_CUDA(cudaEventRecord(c->ev_k0, c->stream));
    const cudaError_t e = launch_coordtime(P, o->prec == KERR_FP32_KAHAN ? 1 : 0, c->sms,
                                           c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ECUDA, "kerr_trace_coordtime: launch failed: %s", cudaGetErrorString(e));
    }
    KERR_CUDA(cudaEventRecord(c->ev_k1, c->stream));
    KERR_CUDA(cudaEventRecord(c->ev_out, c->stream));
    KERR_CUDA(cudaStreamWaitEvent(us, c->ev_out, 0));
    c->have_stats = true;
    c->last_f32 = 0;
    c->last_variant = -1;
    return KERR_OK;
}

int kerr::build_cams(const kerr_camera *cams, int32_t ncam, CamDev *out, int64_t *n_out)
{
    if (!cams || ncam <= 0)
        return fail(KERR_EINVAL, "need at least one camera (ncam = %d)", ncam);
    int64_t n = 0;
    for (int i = 0; i < ncam; ++i) {
        const kerr_camera &k = cams[i];
        if (!(std::fabs(k.a) <= 1.0))
            return fail(KERR_EINVAL, "camera %d: spin %g outside [-1, 1]", i, k.a);
        if (k.nx <= 0 || k.ny <= 0)
            return fail(KERR_EINVAL, "camera %d: size %d x %d", i, k.nx, k.ny);
        if (!(k.half_width > 0.0) || !std::isfinite(k.half_width))
            return fail(KERR_EINVAL, "camera %d: half width %g", i, k.half_width);
        const double rh = 1.0 + std::sqrt(std::max(0.0, 1.0 - k.a * k.a));
        if (!(k.r_obs > 1.01 * rh) || !std::isfinite(k.r_obs) || !std::isfinite(k.incl))
            return fail(KERR_EINVAL, "camera %d: r_obs %g / incl %g invalid", i, k.r_obs, k.incl);
        out[i] = CamDev{k.a, std::sin(k.incl), std::cos(k.incl), k.r_obs, k.half_width, k.nx, k.ny,
                        n};
        n += (int64_t)k.nx * k.ny;
    }
    *n_out = n;
    return KERR_OK;
}

extern "C" int kerr_trace_camera(kerr_ctx *c, const kerr_camera *cams, int32_t ncam,
                                 const kerr_opts *o, double *x_out, double *k_out, int32_t *status,
                                 int32_t *steps, float *diag, float *cross, void *stream)
{
    std::vector<CamDev> cd(std::max(ncam, 1));
    int64_t n = 0;
    int rc = build_cams(cams, ncam, cd.data(), &n);
    if (rc)
        return rc;
    return trace_common(c, MODE_CAMERA, nullptr, nullptr, nullptr, n, cd.data(), ncam, o, x_out,
                        k_out, status, steps, diag, cross, stream);
}

extern "C" int kerr_trace_points(kerr_ctx *c, const double *points, int64_t n, double r_obs,
                                 const kerr_opts *o, double *x_out, double *k_out,
                                 int32_t *status, int32_t *steps, float *diag, float *cross,
                                 void *stream)
{
    if (!(r_obs > 0.0) || !std::isfinite(r_obs))
        return fail(KERR_EINVAL, "r_obs = %g must be finite and > 0", r_obs);
    TraceExtra X;
    X.points = points;
    X.r_obs = r_obs;
    return trace_common(c, MODE_POINTS, nullptr, nullptr, nullptr, n, nullptr, 0, o, x_out, k_out,
                        status, steps, diag, cross, stream, X);
}

// Camera tracing of a device-side list of pixels (the surrogate's fallback):
// geodesic id traces pixel index[id] of cam; n_dev (device) holds how many
// of the capacity n are live.  Outputs are compact (indexed by id).
int kerr_trace_camera_list(kerr_ctx *c, const kerr_camera *cam, const int64_t *index,
                           const unsigned long long *n_dev, int64_t capacity, const kerr_opts *o,
                           double *x_out, double *k_out, int32_t *status, int32_t *steps,
                           float *diag, float *cross, void *stream)
{
    CamDev cd[1];
    int64_t n = 0;
    int rc = build_cams(cam, 1, cd, &n);
    if (rc)
        return rc;
    TraceExtra X;
    X.index = index;
    X.n_dev = n_dev;
    return trace_common(c, MODE_CAMERA, nullptr, nullptr, nullptr, capacity, cd, 1, o,
                        x_out, k_out, status, steps, diag, cross, stream, X);
}

extern "C" int kerr_trace_camera_pixels(kerr_ctx *c, const kerr_camera *cam, const int64_t *index,
                                        int64_t n, const kerr_opts *o, double *x_out,
                                        double *k_out, int32_t *status, int32_t *steps,
                                        float *diag, float *cross, void *stream)
{
    if (n < 0)
        return fail(KERR_EINVAL, "kerr_trace_camera_pixels: n = %lld < 0", (long long)n);
    if (n > 0 && (!index || !is_device_ptr(index)))
        return fail(KERR_EINVAL, "kerr_trace_camera_pixels: index must be device memory");
    return kerr_trace_camera_list(c, cam, index, nullptr, n, o, x_out, k_out, status, steps, diag,
                                  cross, stream);
}

extern "C" int kerr_get_stats(kerr_ctx *c, kerr_stats *out)
{
    if (!c || !out)
        return fail(KERR_EINVAL, "kerr_get_stats: NULL argument");
    std::memset(out, 0, sizeof *out);
    if (!c->have_stats)
        return KERR_OK;
    KERR_CUDA(cudaStreamSynchronize(c->stream));
    unsigned long long h[kScratchWords];
    KERR_CUDA(cudaMemcpy(h, c->d_scratch, sizeof h, cudaMemcpyDeviceToHost));
    const unsigned long long *s = h + 1;
    out->geodesics = (int64_t)s[SC_GEODESICS];
    out->attempts = (int64_t)s[SC_ATTEMPTS];
    out->accepted = (int64_t)s[SC_ACCEPTED];
    out->rhs_fp32 = (int64_t)s[SC_RHS32];
    out->rhs_fp64 = (int64_t)s[SC_RHS64];
    out->attempts_fp64 = (int64_t)s[SC_ATT64];
    out->deferred = (int64_t)s[SC_DEFERRED];
    out->requeued = (int64_t)s[SC_REQUEUED];
    out->queue_errors = (int64_t)s[SC_STATUS + ST_NONE];
    out->rhs_fp32_zone_phase = (int64_t)s[SC_RHS32_ZONE];
    out->attempts_fp32_zone_phase = (int64_t)s[SC_ATT32_ZONE];
    out->clips = (int64_t)s[SC_CLIPS];
    out->clip_rhs = (int64_t)s[SC_CLIP_RHS];
    for (int j = 0; j < 8; ++j)
        out->status_count[j] = (int64_t)s[SC_STATUS + j];
    float ms = 0.f;
    KERR_CUDA(cudaEventElapsedTime(&ms, c->ev_k0, c->ev_k1));
    out->kernel_ms = ms;
    out->variant = c->last_variant;
    if (c->last_f32) {
        float t[4] = {0.f, 0.f, 0.f, 0.f};
        KERR_CUDA(cudaEventElapsedTime(&t[0], c->ev_k0, c->ev_ph[0]));
        KERR_CUDA(cudaEventElapsedTime(&t[1], c->ev_ph[0], c->ev_ph[1]));
        KERR_CUDA(cudaEventElapsedTime(&t[2], c->ev_ph[1], c->ev_ph[2]));
        KERR_CUDA(cudaEventElapsedTime(&t[3], c->ev_ph[2], c->ev_k1));
        for (int i = 0; i < 4; ++i)
            out->phase_ms[i] = t[i];
    } else {
        out->phase_ms[1] = ms;
    }
    return KERR_OK;
}

// ---------------------------------------------------------------------------
// Autotuner (the analogue of the paper's run-time tuning of the work-group
// size, Sec. 4): stepping variants (block size x register cap x geodesics
// per thread x right-hand-side mode), then zone-phase variants with the
// chosen stepping variant, each timed on a sample of the workload; results
// optionally kept in a cache file keyed by GPU, workload shape and precision.
// ---------------------------------------------------------------------------
namespace {

uint32_t fnv1a_bytes(const void *data, size_t bytes, uint32_t h = 2166136261u)
{
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < bytes; ++i) {
        h ^= p[i];
        h *= 16777619u;
    }
    return h;
}

// Name of the current GPU with its SM count, e.g. "NVIDIA GB300 (152 SMs)".
int gpu_label(char *buf, size_t cap)
{
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ECUDA, "autotune: cannot query the device");
    }
    std::snprintf(buf, cap, "%s (%d SMs)", prop.name, prop.multiProcessorCount);
    return KERR_OK;
}

void options_key(const kerr_opts *o, char *buf, size_t cap)
{
    std::snprintf(buf, cap, "prec=%d:tol=%.3g:zone=%.3g:zprec=%d:renorm=%d", o->prec, o->tol,
                  o->prec == KERR_FP32_KAHAN ? o->fp64_zone : 0.0, o->zone_prec, o->renorm_every);
}

// Field separators of the cache file must not occur inside a field.
bool clean_field(const char *s)
{
    for (; *s; ++s)
        if (*s == '\t' || *s == '\n' || *s == '\r')
            return false;
    return true;
}

// Times the candidates with `run(variant, zone_variant)` (which traces the
// sample and returns KERR_OK) and the stats' kernel_ms: one untimed call per
// candidate (graph capture, buffers), then the minimum of `reps` timed ones.
template <typename Run>
int sweep(kerr_ctx *c, const kerr_opts *o, int reps, Run run, kerr_tuning *t)
{
    const int prec = o->prec;
    auto time_one = [&](int v, int zv, float *ms) -> int {
        float best = 1e30f;
        for (int rep = 0; rep <= reps; ++rep) {
            int rc = run(v, zv);
            if (rc)
                return rc;
            kerr_stats st;
            rc = kerr_get_stats(c, &st);
            if (rc)
                return rc;
            if (rep > 0)
                best = std::min(best, st.kernel_ms);
        }
        *ms = best;
        return KERR_OK;
    };
    const bool zone = prec == KERR_FP32_KAHAN && o->fp64_zone > 0.0;
    const int zdef = zone ? kDefaultZoneVariant : -1;
    int best_v = kDefaultVariant[prec];
    float best_ms = 1e30f;
    t->timed = 0;
    for (int v = 0; v < kNumVariants; ++v) {
        if (prec == KERR_FP64 && kVariantRays[v] != 1)
            continue;                       // two geodesics per thread: FP32 only
        float ms = 0.f;
        int rc = time_one(v, zdef, &ms);
        if (rc)
            return rc;
        ++t->timed;
        if (ms < best_ms) {
            best_ms = ms;
            best_v = v;
        }
    }
    int best_z = zdef;
    if (zone) {
        for (int zv = 0; zv < kNumZoneVariants; ++zv) {
            if (zv == zdef)
                continue;                   // timed with the stepping variants
            float ms = 0.f;
            int rc = time_one(best_v, zv, &ms);
            if (rc)
                return rc;
            ++t->timed;
            if (ms < best_ms) {
                best_ms = ms;
                best_z = zv;
            }
        }
    }
    t->variant = best_v;
    t->zone_variant = best_z;
    t->ms = best_ms;
    t->from_cache = 0;
    c->tuned[prec] = best_v;
    c->tuned_zone[prec] = best_z;
    return KERR_OK;
}

struct DevBufs {
    std::vector<void *> p;
    ~DevBufs()
    {
        for (void *q : p)
            cudaFree(q);
    }
    template <typename T> cudaError_t get(T **out, size_t bytes)
    {
        void *q = nullptr;
        cudaError_t e = dev_alloc(&q, bytes);
        if (e == cudaSuccess)
            p.push_back(q);
        *out = (T *)q;
        return e;
    }
};

// Looks the workload up in the cache (when a path is given); on a hit applies
// the stored choice to the context.
int cache_hit(kerr_ctx *c, const kerr_opts *o, const char *path, const char *key,
              kerr_tuning *out, bool *hit)
{
    *hit = false;
    if (!path)
        return KERR_OK;
    char gpu[256];
    int rc = gpu_label(gpu, sizeof gpu);
    if (rc)
        return rc;
    rc = kerr_tune_cache_lookup(path, gpu, key, out);
    if (rc < 0)
        return rc;
    if (rc == KERR_OK) {
        const bool zone = o->prec == KERR_FP32_KAHAN && o->fp64_zone > 0.0;
        if (out->variant < 0 || out->variant >= kNumVariants ||
            (o->prec == KERR_FP64 && kVariantRays[out->variant] != 1) ||
            out->zone_variant >= kNumZoneVariants || (zone && out->zone_variant < 0))
            return fail(KERR_EINVAL, "autotune cache: stored configuration is out of range");
        c->tuned[o->prec] = out->variant;
        c->tuned_zone[o->prec] = zone ? out->zone_variant : -1;
        out->from_cache = 1;
        *hit = true;
    }
    return KERR_OK;
}

int cache_store(const char *path, const char *key, const kerr_tuning *t)
{
    if (!path)
        return KERR_OK;
    char gpu[256];
    int rc = gpu_label(gpu, sizeof gpu);
    if (rc)
        return rc;
    return kerr_tune_cache_store(path, gpu, key, t);
}

} // namespace

extern "C" int kerr_tune_cache_lookup(const char *path, const char *gpu, const char *key,
                                      kerr_tuning *out)
{
    if (!path || !gpu || !key || !out)
        return fail(KERR_EINVAL, "kerr_tune_cache_lookup: NULL argument");
    FILE *f = std::fopen(path, "r");
    if (!f)
        return 1;                           // no cache yet: a miss
    char line[1024];
    bool found = false;
    kerr_tuning t;
    std::memset(&t, 0, sizeof t);
    int lineno = 0;
    while (std::fgets(line, sizeof line, f)) {
        ++lineno;
        const size_t len = std::strlen(line);
        if (len == 0 || line[0] == '#' || line[0] == '\n')
            continue;
        if (line[len - 1] != '\n' && !std::feof(f)) {
            std::fclose(f);
            return fail(KERR_EINVAL, "kerr_tune_cache_lookup: line %d too long", lineno);
        }
        // gpu \t key \t variant \t zone_variant \t ms
        char *fields[5];
        int nf = 0;
        char *p = line;
        fields[nf++] = p;
        for (; *p && nf < 5; ++p)
            if (*p == '\t') {
                *p = '\0';
                fields[nf++] = p + 1;
            }
        int v = 0, zv = 0;
        float ms = 0.f;
        if (nf != 5 || std::sscanf(fields[2], "%d", &v) != 1 ||
            std::sscanf(fields[3], "%d", &zv) != 1 || std::sscanf(fields[4], "%f", &ms) != 1) {
            std::fclose(f);
            return fail(KERR_EINVAL, "kerr_tune_cache_lookup: malformed line %d", lineno);
        }
        if (std::strcmp(fields[0], gpu) == 0 && std::strcmp(fields[1], key) == 0) {
            t.variant = v;                  // the last matching line wins
            t.zone_variant = zv;
            t.ms = ms;
            found = true;
        }
    }
    std::fclose(f);
    if (!found)
        return 1;
    t.from_cache = 1;
    *out = t;
    return KERR_OK;
}

extern "C" int kerr_tune_cache_store(const char *path, const char *gpu, const char *key,
                                     const kerr_tuning *t)
{
    if (!path || !gpu || !key || !t)
        return fail(KERR_EINVAL, "kerr_tune_cache_store: NULL argument");
    if (!clean_field(gpu) || !clean_field(key) || !*gpu || !*key)
        return fail(KERR_EINVAL, "kerr_tune_cache_store: empty field or tab/newline in a field");
    FILE *f = std::fopen(path, "a");
    if (!f)
        return fail(KERR_EINVAL, "kerr_tune_cache_store: cannot open the cache file");
    const int n = std::fprintf(f, "%s\t%s\t%d\t%d\t%.6g\n", gpu, key, t->variant,
                               t->zone_variant, (double)t->ms);
    const bool closed = std::fclose(f) == 0;
    if (n < 0 || !closed)
        return fail(KERR_EINVAL, "kerr_tune_cache_store: write failed");
    return KERR_OK;
}

extern "C" int kerr_tune_key_cameras(const kerr_camera *cams, int32_t ncam, const kerr_opts *o,
                                     char *buf, int32_t cap)
{
    if (!cams || ncam < 1 || !o || !buf || cap < 1)
        return fail(KERR_EINVAL, "kerr_tune_key_cameras: bad argument");
    int64_t n = 0;
    uint32_t h = 2166136261u;
    for (int i = 0; i < ncam; ++i) {
        const kerr_camera &k = cams[i];
        n += (int64_t)k.nx * k.ny;
        const double d[4] = {k.a, k.incl, k.r_obs, k.half_width};
        const int32_t w[2] = {k.nx, k.ny};
        h = fnv1a_bytes(d, sizeof d, h);
        h = fnv1a_bytes(w, sizeof w, h);
    }
    char ok[160];
    options_key(o, ok, sizeof ok);
    const int m = std::snprintf(buf, (size_t)cap, "cameras:ncam=%d:rays=%lld:geom=%08x:%s", ncam,
                                (long long)n, h, ok);
    if (m < 0 || m >= cap)
        return fail(KERR_EINVAL, "kerr_tune_key_cameras: buffer too small");
    return KERR_OK;
}

extern "C" int kerr_tune_key_particles(int64_t n, const kerr_opts *o, char *buf, int32_t cap)
{
    if (n < 1 || !o || !buf || cap < 1)
        return fail(KERR_EINVAL, "kerr_tune_key_particles: bad argument");
    char ok[160];
    options_key(o, ok, sizeof ok);
    const int m = std::snprintf(buf, (size_t)cap, "particles:n=%lld:max_steps=%lld:%s",
                                (long long)n, (long long)o->max_steps, ok);
    if (m < 0 || m >= cap)
        return fail(KERR_EINVAL, "kerr_tune_key_particles: buffer too small");
    return KERR_OK;
}

extern "C" int kerr_autotune_cameras(kerr_ctx *c, const kerr_camera *cams, int32_t ncam,
                                     const kerr_opts *o, int64_t sample, const char *cache_path,
                                     kerr_tuning *out, void *stream)
{
    if (!c || !cams || !out)
        return fail(KERR_EINVAL, "kerr_autotune_cameras: NULL argument");
    int rc = check_opts(o);
    if (rc)
        return rc;
    std::vector<CamDev> cd(std::max(ncam, 1));
    int64_t n = 0;
    rc = build_cams(cams, ncam, cd.data(), &n);
    if (rc)
        return rc;
    char key[512];
    rc = kerr_tune_key_cameras(cams, ncam, o, key, sizeof key);
    if (rc)
        return rc;
    bool hit = false;
    rc = cache_hit(c, o, cache_path, key, out, &hit);
    if (rc || hit)
        return rc;
    if (sample < 1024)
        sample = 1024;
    // each camera at a lower resolution over the same field of view, its
    // share of the sample in proportion to its rays
    std::vector<kerr_camera> sub(cams, cams + ncam);
    int64_t m = 0;
    for (auto &k : sub) {
        const double share = (double)sample * ((double)k.nx * k.ny) / (double)n;
        const double f = std::min(1.0, std::sqrt(share / ((double)k.nx * k.ny)));
        k.nx = std::max(1, std::min(k.nx, (int)std::lround(k.nx * f)));
        k.ny = std::max(1, std::min(k.ny, (int)std::lround(k.ny * f)));
        m += (int64_t)k.nx * k.ny;
    }
    DevBufs B;
    double *xo = nullptr, *ko = nullptr;
    int32_t *so = nullptr, *no = nullptr;
    cudaError_t e = B.get(&xo, 4 * m * sizeof(double));
    if (e == cudaSuccess)
        e = B.get(&ko, 4 * m * sizeof(double));
    if (e == cudaSuccess)
        e = B.get(&so, m * sizeof(int32_t));
    if (e == cudaSuccess)
        e = B.get(&no, m * sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ENOMEM, "kerr_autotune_cameras: allocation failed");
    }
    kerr_opts oo = *o;
    rc = sweep(c, o, 2,
               [&](int v, int zv) {
                   oo.variant = v;
                   oo.zone_variant = zv;
                   return kerr_trace_camera(c, sub.data(), ncam, &oo, xo, ko, so, no, nullptr,
                                            nullptr, stream);
               },
               out);
    cudaStreamSynchronize(c->stream);
    if (rc)
        return rc;
    return cache_store(cache_path, key, out);
}

extern "C" int kerr_autotune_particles(kerr_ctx *c, const double *x0, const double *v0,
                                       const double *t_end, int64_t n, const kerr_opts *o,
                                       int64_t sample, const char *cache_path, kerr_tuning *out,
                                       void *stream)
{
    if (!c || !x0 || !v0 || !out)
        return fail(KERR_EINVAL, "kerr_autotune_particles: NULL argument");
    int rc = check_opts(o);
    if (rc)
        return rc;
    if (n < 1)
        return fail(KERR_EINVAL, "kerr_autotune_particles: n = %lld < 1", (long long)n);
    char key[512];
    rc = kerr_tune_key_particles(n, o, key, sizeof key);
    if (rc)
        return rc;
    bool hit = false;
    rc = cache_hit(c, o, cache_path, key, out, &hit);
    if (rc || hit)
        return rc;
    if (sample < 256)
        sample = 256;
    const int64_t stride = std::max<int64_t>(1, n / sample);
    const int64_t m = std::min<int64_t>(sample, (n + stride - 1) / stride);
    DevBufs B;
    double *xs = nullptr, *vs = nullptr, *ts = nullptr, *xo = nullptr, *ko = nullptr;
    int32_t *so = nullptr, *no = nullptr;
    cudaError_t e = B.get(&xs, 4 * m * sizeof(double));
    if (e == cudaSuccess)
        e = B.get(&vs, 3 * m * sizeof(double));
    if (e == cudaSuccess && t_end)
        e = B.get(&ts, m * sizeof(double));
    if (e == cudaSuccess)
        e = B.get(&xo, 4 * m * sizeof(double));
    if (e == cudaSuccess)
        e = B.get(&ko, 4 * m * sizeof(double));
    if (e == cudaSuccess)
        e = B.get(&so, m * sizeof(int32_t));
    if (e == cudaSuccess)
        e = B.get(&no, m * sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ENOMEM, "kerr_autotune_particles: allocation failed");
    }
    // every stride-th particle of each plane (the planes may be host or
    // device memory)
    auto gather = [&](double *dst, const double *src, int planes) -> cudaError_t {
        for (int j = 0; j < planes; ++j) {
            cudaError_t ee = cudaMemcpy2DAsync(dst + j * m, sizeof(double), src + j * n,
                                               (size_t)stride * sizeof(double), sizeof(double),
                                               (size_t)m, cudaMemcpyDefault, c->stream);
            if (ee != cudaSuccess)
                return ee;
        }
        return cudaSuccess;
    };
    e = gather(xs, x0, 4);
    if (e == cudaSuccess)
        e = gather(vs, v0, 3);
    if (e == cudaSuccess && t_end)
        e = gather(ts, t_end, 1);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ECUDA, "kerr_autotune_particles: sample gather failed: %s",
                    cudaGetErrorString(e));
    }
    kerr_opts oo = *o;
    rc = sweep(c, o, 1,
               [&](int v, int zv) {
                   oo.variant = v;
                   oo.zone_variant = zv;
                   return kerr_trace_particles(c, xs, vs, ts, m, &oo, xo, ko, so, no, nullptr,
                                               nullptr, stream);
               },
               out);
    cudaStreamSynchronize(c->stream);
    if (rc)
        return rc;
    return cache_store(cache_path, key, out);
}

extern "C" int kerr_autotune(kerr_ctx *c, const kerr_camera *cam, const kerr_opts *o,
                             int64_t sample, int32_t *best, void *stream)
{
    if (!c || !cam || !best)
        return fail(KERR_EINVAL, "kerr_autotune: NULL argument");
    kerr_tuning t;
    const int rc = kerr_autotune_cameras(c, cam, 1, o, sample, nullptr, &t, stream);
    if (rc)
        return rc;
    *best = t.variant;
    return KERR_OK;
}
