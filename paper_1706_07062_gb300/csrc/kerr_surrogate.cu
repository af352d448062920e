// kerr_surrogate.cu -- the learned surrogate of the geodesic integrator:
// network object, training (forward, loss, backward, Adam), inference, and
// rendering with an integrator fallback near the shadow edge.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/kerr.h"
#define KERR_TYPES_ONLY
#include "kerr_trace.cuh"
#include "kerr_mlp.cuh"
#include "kerr_variants.h"

using namespace kerr;
using namespace kerr::mlp;
using bf16 = __nv_bfloat16;

// Camera tracing of a device-side pixel list (kerr_api.cu).
int kerr_trace_camera_list(kerr_ctx *c, const kerr_camera *cam, const int64_t *index,
                           const unsigned long long *n_dev, int64_t capacity, const kerr_opts *o,
                           double *x_out, double *k_out, int32_t *status, int32_t *steps,
                           float *diag, float *cross, void *stream);

namespace {

int fail(int code, const char *msg) { return kerr_set_error(code, msg); }

#define SURR_CUDA(call)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            cudaGetLastError();                                                                \
            return fail(KERR_ECUDA, #call " failed");                                          \
        }                                                                                      \
    } while (0)

// Parameter layout: for l = 0..4, W_l [out][in] then b_l [out].
struct Layout {
    size_t w[kLayers], b[kLayers], total;
    Layout()
    {
        size_t o = 0;
        for (int l = 0; l < kLayers; ++l) {
            w[l] = o;
            o += (size_t)out_dim(l) * in_dim(l);
            b[l] = o;
            o += out_dim(l);
        }
        total = o;
    }
};
const Layout kL;

struct WOffsets {
    int64_t w[kLayers];
    int64_t end;
};
WOffsets woffsets()
{
    WOffsets o;
    for (int l = 0; l < kLayers; ++l)
        o.w[l] = (int64_t)kL.w[l];
    o.end = (int64_t)kL.total;
    return o;
}

// ---------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------
__global__ void to_bf16_kernel(const float *__restrict__ src, bf16 *__restrict__ dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16(src[i]);
}

// Step k's values; sched[k] = (learning rate, Adam bias corrections) from
// the host (cosine schedule, 1 / (1 - beta^t)).
__global__ void train_step_kernel(StepCtl *ctl, const float3 *__restrict__ sched,
                                  long long steps_per_epoch, long long batch)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    const long long k = ctl->k;
    ctl->r0 = (k % steps_per_epoch) * batch;
    ctl->ep = (int)(k / steps_per_epoch);
    const float3 v = sched[k];
    ctl->lr = v.x;
    ctl->c1 = v.y;
    ctl->c2 = v.z;
    ctl->k = k + 1;
}

// Network input rows [n][16] (bf16, 4 live) from in [n][4]; with A0T also
// the transposed copy [16][ldT] (training: the batch-contracted operand of
// the first layer's weight gradient).
__global__ void input_kernel(const float *__restrict__ in, bf16 *__restrict__ A0, int64_t n,
                             bf16 *__restrict__ A0T = nullptr, int64_t ldT = 0,
                             const StepCtl *__restrict__ ctl = nullptr)
{
    if (ctl)
        in += ctl->r0 * kIn;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * kInPad;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / kInPad;
        const int c = (int)(i % kInPad);
        const bf16 v = __float2bfloat16(c < kIn ? in[r * kIn + c] : 0.0f);
        A0[i] = v;
        if (A0T)
            A0T[c * ldT + r] = v;
    }
}

// Loss and output gradient.  out [n][64] fp32 (8 live), targets/mask [n][8].
// Loss row = softplus(o0) - y0 o0 + sum_{j>=1} m_j (o_j - y_j)^2; the
// gradient of the batch mean goes to dOut [n][64] (bf16, padding zero).
__global__ void loss_kernel(const float *__restrict__ out, const float *__restrict__ tgt,
                            const float *__restrict__ msk, int64_t n, float inv_n,
                            bf16 *__restrict__ dOut, float *__restrict__ loss_sum,
                            bf16 *__restrict__ dOutT, int64_t ldT,
                            const StepCtl *__restrict__ ctl = nullptr)
{
    if (ctl) {
        tgt += ctl->r0 * kOut;
        msk += ctl->r0 * kOut;
        loss_sum += ctl->ep;
    }
    float local = 0.0f;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const float *o = out + r * kOutPad;
        const float *y = tgt + r * kOut;
        const float *m = msk + r * kOut;
        const float z = o[0];
        const float sp = z > 0.f ? z + log1pf(__expf(-z)) : log1pf(__expf(z));
        local += sp - y[0] * z;
        const float sig = 1.0f / (1.0f + __expf(-z));
        __align__(16) bf16 dv[kOut];
        dv[0] = __float2bfloat16((sig - y[0]) * inv_n);
#pragma unroll
        for (int j = 1; j < kOut; ++j) {
            const float e = m[j] * (o[j] - y[j]);
            local += e * (o[j] - y[j]);
            dv[j] = __float2bfloat16(2.0f * e * inv_n);
        }
        // the row's 64 gradient entries (8 live) as eight 16-byte stores
        uint4 *d = reinterpret_cast<uint4 *>(dOut + r * kOutPad);
        d[0] = *reinterpret_cast<const uint4 *>(dv);
#pragma unroll
        for (int q = 1; q < kOutPad / 8; ++q)
            d[q] = make_uint4(0u, 0u, 0u, 0u);
        if (dOutT) {
#pragma unroll
            for (int j = 0; j < kOut; ++j)
                dOutT[j * ldT + r] = dv[j];     // rows 8..63 of dOutT stay zero
        }
    }
    // block reduction
    __shared__ float red[32];
    for (int o2 = 16; o2 > 0; o2 >>= 1)
        local += __shfl_xor_sync(0xffffffffu, local, o2);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o2 = 16; o2 > 0; o2 >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o2);
        if (threadIdx.x == 0)
            atomicAdd(loss_sum, v * inv_n);
    }
}

// Column sums of a bf16 [n][w] matrix into db (output-layer bias gradient).
__global__ void colsum_kernel(const bf16 *__restrict__ X, int64_t n, int w, float *__restrict__ db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= w)
        return;
    float s = 0.0f;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y)
        s += __bfloat162float(X[r * w + c]);
    atomicAdd(&db[c], s);
}

// Transposed bf16 copy of every weight matrix: layer l's W [out][in] at the
// same offset as [in][out] (the B operand of the input-gradient GEMMs).
__global__ void transpose_weights_kernel(const bf16 *__restrict__ wbf, bf16 *__restrict__ wt,
                                         WOffsets o)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < o.end;
         i += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < kLayers && i >= o.w[l + 1])
            ++l;
        const int64_t j = i - o.w[l];
        if (j >= (int64_t)out_dim(l) * in_dim(l))
            continue;                               // bias entries
        const int K = in_dim(l), N = out_dim(l);
        const int nrow = (int)(j / K), k = (int)(j % K);
        wt[o.w[l] + (int64_t)k * N + nrow] = wbf[i];
    }
}

// Adam on the whole parameter vector; refreshes the bf16 copy of each weight.
// The transposed bf16 copy (see transpose_weights_kernel) is written in the
// same pass; learning rate and bias corrections come from the step control.
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, bf16 *__restrict__ wbf,
                            bf16 *__restrict__ wbfT, WOffsets o, int64_t n,
                            const StepCtl *__restrict__ ctl, float b1, float b2, float eps)
{
    const float lr = ctl->lr, c1 = ctl->c1, c2 = ctl->c2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        w[i] = wi;
        const bf16 wb = __float2bfloat16(wi);
        wbf[i] = wb;
        int l = 0;
        while (l + 1 < kLayers && i >= o.w[l + 1])
            ++l;
        const int64_t j = i - o.w[l];
        if (j < (int64_t)out_dim(l) * in_dim(l)) {            // weights, not biases
            const int K = in_dim(l), N = out_dim(l);
            wbfT[o.w[l] + (j % K) * N + j / K] = wb;
        }
    }
}

int grid_1d(int64_t n, int block = 256)
{
    int64_t g = (n + block - 1) / block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

// C = A B^T with epilogue EPI on the tensor cores (kerr_gemm_tc.cu); a
// pipeline wait that gives up sets *err (checked after the call).
template <int EPI>
cudaError_t gemm(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K, EpiArgs e,
                 unsigned *err, cudaStream_t s, int splits = 1)
{
    return gemm_tc(A, lda, B, ldb, M, N, K, EPI, e, splits, err, s);
}

// Split count for a weight gradient contracted over `rows` batch rows: about
// four 64-row slices per CTA, so that the four 128 x 128 output tiles of a
// hidden layer spread over ~128 CTAs (each adds its partial tile with
// coalesced atomics).
int wsplits(int64_t rows) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, rows / 256)); }

} // namespace

// Grow-only device scratch of kerr_surrogate_render (kept by the surrogate,
// so that a render allocates nothing once the sizes are reached).
struct RenderScratch {
    int64_t cap_n = 0, cap_m = 0;
    float *in = nullptr, *o = nullptr;
    int64_t *idx = nullptr;
    float2 *curve = nullptr;
    double *rint = nullptr;
    float4 *bounds = nullptr;
    unsigned long long *cnt = nullptr;
    double *x = nullptr, *k = nullptr;
    int32_t *stat = nullptr, *nst = nullptr;
    float *crs = nullptr;
};
constexpr int kCurveSamples = 2048;   // per branch

static void free_render(RenderScratch &r)
{
    cudaFree(r.in);
    cudaFree(r.o);
    cudaFree(r.idx);
    cudaFree(r.curve);
    cudaFree(r.rint);
    cudaFree(r.bounds);
    cudaFree(r.cnt);
    cudaFree(r.x);
    cudaFree(r.k);
    cudaFree(r.stat);
    cudaFree(r.nst);
    cudaFree(r.crs);
    r = RenderScratch();
}

// ===========================================================================
// the surrogate object
// ===========================================================================
struct kerr_surrogate {
    int device = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // fp32 [total]
    bf16 *wbf = nullptr;                                           // bf16 copy [total]
    int64_t step = 0;
    // activations for a batch of `cap` rows
    int64_t cap = 0;
    bf16 *A[kLayers] = {};        // layer inputs (A[0]: [cap][16]; others [cap][256])
    float *Z[kLayers - 1] = {};   // hidden pre-activations [cap][256]
    float *out = nullptr;         // [cap][64]
    bf16 *dOut = nullptr;         // [cap][64]
    bf16 *dZ[2] = {};             // [cap][256] hidden-layer gradients (two layers in flight)
    // transposed batch operands of the weight gradients (row stride ldT,
    // columns >= the batch's rows kept zero): AT[l] = A[l]^T [in_dim(l)][ldT],
    // DT[i] = dZ[i]^T [256][ldT], OT = dOut^T [64][ldT]
    bf16 *AT[kLayers] = {};
    bf16 *DT[2] = {};
    bf16 *OT = nullptr;
    int64_t ldT = 0;
    bf16 *wbfT = nullptr;         // transposed bf16 weights (same offsets)
    float *loss = nullptr;        // [1]
    RenderScratch *render = nullptr;   // kerr_surrogate_render's scratch
    bf16 *wpk = nullptr;          // weights in the tensor-core operand layout
    unsigned *tc_err = nullptr;   // fused forward: a pipeline wait gave up
    int sms = 0;
    // fused training (kerr_train_tc.cu): batch buffers of tb.cap rows and the
    // packed training weights (valid unless the GEMM path's Adam ran last)
    TrainBufs tb{};
    bf16 *wtp = nullptr;
    bool wtp_valid = false;
    float *part = nullptr;        // the gradient's partial sums over batch splits
    bool wbfT_valid = true;       // the transposed bf16 copy (the fused Adam skips it)
};

static void free_train(kerr_surrogate *s)
{
    cudaFree(s->tb.sp);
    cudaFree(s->tb.ht);
    cudaFree(s->tb.dt);
    s->tb = TrainBufs{};
}

// Batch buffers of the fused training kernels for `rows` rows (capacity a
// multiple of 128, grow-only); the never-written parts are zeroed once.
static int ensure_train(kerr_surrogate *s, int64_t rows)
{
    const int64_t cap = (rows + 127) / 128 * 128;
    if (cap <= s->tb.cap)
        return KERR_OK;
    free_train(s);
    TrainBufs b{};
    b.cap = cap;
    cudaError_t e = dev_alloc(&b.sp, train_sp_elems(cap) * sizeof(float));
    if (e == cudaSuccess)
        e = dev_alloc(&b.ht, train_ht_elems(cap) * sizeof(bf16));
    if (e == cudaSuccess)
        e = dev_alloc(&b.dt, train_dt_elems(cap) * sizeof(bf16));
    if (e == cudaSuccess)
        e = train_zero_bufs(b, 0);
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b.sp);
        cudaFree(b.ht);
        cudaFree(b.dt);
        return fail(KERR_ENOMEM, "surrogate: training buffers");
    }
    s->tb = b;
    return KERR_OK;
}

static void free_batch(kerr_surrogate *s)
{
    for (int l = 0; l < kLayers; ++l)
        cudaFree(s->A[l]), s->A[l] = nullptr;
    for (int l = 0; l < kLayers - 1; ++l)
        cudaFree(s->Z[l]), s->Z[l] = nullptr;
    cudaFree(s->out);
    cudaFree(s->dOut);
    for (int i = 0; i < 2; ++i) {
        cudaFree(s->dZ[i]), s->dZ[i] = nullptr;
        cudaFree(s->DT[i]), s->DT[i] = nullptr;
    }
    for (int l = 0; l < kLayers; ++l)
        cudaFree(s->AT[l]), s->AT[l] = nullptr;
    cudaFree(s->OT);
    s->OT = nullptr;
    s->ldT = 0;
    s->out = nullptr;
    s->dOut = nullptr;
    s->cap = 0;
}

static int ensure_batch(kerr_surrogate *s, int64_t rows, bool training)
{
    if (rows <= s->cap && (!training || s->Z[0]))
        return KERR_OK;
    free_batch(s);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l)
        e = dev_alloc(&s->A[l], (size_t)rows * in_dim(l) * sizeof(bf16));
    if (e == cudaSuccess)
        e = dev_alloc(&s->out, (size_t)rows * kOutPad * sizeof(float));
    if (training) {
        for (int l = 0; l < kLayers - 1 && e == cudaSuccess; ++l)
            e = dev_alloc(&s->Z[l], (size_t)rows * kHidden * sizeof(float));
        if (e == cudaSuccess)
            e = dev_alloc(&s->dOut, (size_t)rows * kOutPad * sizeof(bf16));
        for (int i = 0; i < 2; ++i)
            if (e == cudaSuccess)
                e = dev_alloc(&s->dZ[i], (size_t)rows * kHidden * sizeof(bf16));
        const int64_t ldT = (rows + 7) / 8 * 8;
        auto zalloc = [&](bf16 **p, int64_t h) {
            if (e == cudaSuccess)
                e = dev_alloc(p, (size_t)h * ldT * sizeof(bf16));
            if (e == cudaSuccess)
                e = cudaMemset(*p, 0, (size_t)h * ldT * sizeof(bf16));
        };
        for (int l = 0; l < kLayers; ++l)
            zalloc(&s->AT[l], in_dim(l));
        zalloc(&s->DT[0], kHidden);
        zalloc(&s->DT[1], kHidden);
        zalloc(&s->OT, kOutPad);
        if (e == cudaSuccess)
            s->ldT = ldT;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_batch(s);
        return fail(KERR_ENOMEM, "surrogate: activation buffers");
    }
    s->cap = rows;
    return KERR_OK;
}

extern "C" int64_t kerr_surrogate_num_params(void) { return (int64_t)kL.total; }

extern "C" int kerr_surrogate_destroy(kerr_surrogate *s)
{
    if (!s)
        return KERR_OK;
    cudaDeviceSynchronize();
    free_batch(s);
    free_train(s);
    cudaFree(s->wtp);
    cudaFree(s->part);
    cudaFree(s->w);
    cudaFree(s->g);
    cudaFree(s->m);
    cudaFree(s->v);
    cudaFree(s->wbf);
    cudaFree(s->wbfT);
    cudaFree(s->loss);
    cudaFree(s->wpk);
    cudaFree(s->tc_err);
    if (s->render) {
        free_render(*s->render);
        delete s->render;
    }
    delete s;
    return KERR_OK;
}

extern "C" int kerr_surrogate_create(const float *init, kerr_surrogate **out)
{
    if (!init || !out)
        return fail(KERR_EINVAL, "kerr_surrogate_create: NULL argument");
    *out = nullptr;
    kerr_surrogate *s = new (std::nothrow) kerr_surrogate();
    if (!s)
        return fail(KERR_ENOMEM, "kerr_surrogate_create: host allocation");
    s->render = new (std::nothrow) RenderScratch();
    if (!s->render) {
        delete s;
        return fail(KERR_ENOMEM, "kerr_surrogate_create: host allocation");
    }
    const size_t n = kL.total;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess)
        e = dev_alloc(&s->w, n * sizeof(float));
    if (e == cudaSuccess)
        e = dev_alloc(&s->g, n * sizeof(float));
    if (e == cudaSuccess)
        e = dev_alloc(&s->m, n * sizeof(float));
    if (e == cudaSuccess)
        e = dev_alloc(&s->v, n * sizeof(float));
    if (e == cudaSuccess)
        e = dev_alloc(&s->wbf, n * sizeof(bf16));
    if (e == cudaSuccess)
        e = dev_alloc(&s->wbfT, n * sizeof(bf16));
    if (e == cudaSuccess)
        e = dev_alloc(&s->loss, sizeof(float));
    if (e == cudaSuccess)
        e = dev_alloc(&s->wpk, packed_weight_elems() * sizeof(bf16));
    if (e == cudaSuccess)
        e = dev_alloc(&s->wtp, train_packed_elems() * sizeof(bf16));
    if (e == cudaSuccess)
        e = dev_alloc(&s->part, train_part_elems(n) * sizeof(float));
    if (e == cudaSuccess)
        e = dev_alloc(&s->tc_err, sizeof(unsigned));
    if (e == cudaSuccess)
        e = cudaMemset(s->tc_err, 0, sizeof(unsigned));
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess)
        e = gemm_tc_prepare();
    if (e == cudaSuccess)
        e = train_prepare();
    if (e == cudaSuccess)
        e = cudaMemcpy(s->w, init, n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(s->g, 0, n * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemset(s->m, 0, n * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemset(s->v, 0, n * sizeof(float));
    if (e == cudaSuccess) {
        to_bf16_kernel<<<grid_1d(n), 256>>>(s->w, s->wbf, n);
        transpose_weights_kernel<<<grid_1d(n), 256>>>(s->wbf, s->wbfT, woffsets());
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = train_pack(s->wbf, kL.w, s->wtp, 0);
    if (e == cudaSuccess)
        s->wtp_valid = true;
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        kerr_surrogate_destroy(s);
        return fail(KERR_ENOMEM, "kerr_surrogate_create: device allocation");
    }
    *out = s;
    return KERR_OK;
}

extern "C" int kerr_surrogate_get_params(kerr_surrogate *s, float *host_out)
{
    if (!s || !host_out)
        return fail(KERR_EINVAL, "kerr_surrogate_get_params: NULL argument");
    SURR_CUDA(cudaDeviceSynchronize());
    SURR_CUDA(cudaMemcpy(host_out, s->w, kL.total * sizeof(float), cudaMemcpyDeviceToHost));
    return KERR_OK;
}

extern "C" int kerr_surrogate_get_grad(kerr_surrogate *s, float *host_out)
{
    if (!s || !host_out)
        return fail(KERR_EINVAL, "kerr_surrogate_get_grad: NULL argument");
    SURR_CUDA(cudaDeviceSynchronize());
    SURR_CUDA(cudaMemcpy(host_out, s->g, kL.total * sizeof(float), cudaMemcpyDeviceToHost));
    return KERR_OK;
}

// Forward pass of `rows` rows already in s->A[0]; keeps pre-activations when
// training.  The final outputs land in s->out [rows][64].
static cudaError_t forward_rows(kerr_surrogate *s, int64_t rows, bool training, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
        const int K = in_dim(l), N = out_dim(l);
        EpiArgs ea;
        std::memset(&ea, 0, sizeof ea);
        ea.bias = s->w + kL.b[l];
        const bf16 *W = s->wbf + kL.w[l];
        if (l < kLayers - 1) {
            ea.Aout = s->A[l + 1];
            ea.lda_out = N;
            if (training) {
                ea.C = s->Z[l];
                ea.ldc = N;
                ea.AoutT = s->AT[l + 1];     // transposed activations for the weight gradient
                ea.ldT = s->ldT;
                e = gemm<EPI_BIAS_SILU>(s->A[l], K, W, K, (int)rows, N, K, ea, s->tc_err, st);
            } else {
                e = gemm<EPI_BIAS_SILU_BF16>(s->A[l], K, W, K, (int)rows, N, K, ea, s->tc_err,
                                             st);
            }
        } else {
            ea.C = s->out;
            ea.ldc = N;
            e = gemm<EPI_BIAS_F32>(s->A[l], K, W, K, (int)rows, N, K, ea, s->tc_err, st);
        }
    }
    return e;
}

// Backward pass after forward_rows(training) and loss_kernel: gradients of
// the batch accumulate into s->g (zeroed first).  Each hidden layer's
// gradient comes out of the previous GEMM's epilogue already multiplied by
// the SiLU derivative, with its transpose and bias gradient.  The weight gradients
// contract over the batch rows, rounded up to a multiple of 8 (the
// transposed operands are zero from `rows` on).
static cudaError_t backward_rows(kerr_surrogate *s, int64_t rows, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(s->g, 0, kL.total * sizeof(float), st);
    const int R = (int)rows;
    const int R8 = (R + 7) / 8 * 8;
    const int64_t LT = s->ldT;
    if (R8 > R) {
        // columns R .. R8-1 of the transposed operands may hold an earlier,
        // larger batch's values
        auto clear_tail = [&](bf16 *p, int h) {
            if (e == cudaSuccess)
                e = cudaMemset2DAsync(p + R, LT * sizeof(bf16), 0, (R8 - R) * sizeof(bf16), h,
                                      st);
        };
        for (int l = 0; l < kLayers; ++l)
            clear_tail(s->AT[l], in_dim(l));
        clear_tail(s->DT[0], kHidden);
        clear_tail(s->DT[1], kHidden);
        clear_tail(s->OT, kOutPad);
    }
    // dW_l [N][K] += D^T A_l over the batch, with DT = D^T [N][LT] and
    // AT[l] = A_l^T [K][LT] written by the producers
    auto weight_grad = [&](const bf16 *DT, int l) {
        const int K = in_dim(l), N = out_dim(l);
        EpiArgs ea;
        std::memset(&ea, 0, sizeof ea);
        ea.C = s->g + kL.w[l];
        ea.ldc = K;
        return gemm<EPI_F32_ATOMIC>(DT, (int)LT, s->AT[l], (int)LT, N, K, R8, ea, s->tc_err, st,
                                    wsplits(rows));
    };
    // gradient into layer l's input through the previous layer's SiLU:
    // dZ_{l-1} = (D W_l) * silu'(Z_{l-1}) with W_l^T [K][N] as the B operand,
    // written to dZ[i] and DT[i] with the bias gradient of layer l - 1
    auto input_grad = [&](const bf16 *D, int l, int i) {
        const int K = in_dim(l), N = out_dim(l);
        EpiArgs eb;
        std::memset(&eb, 0, sizeof eb);
        eb.Zin = s->Z[l - 1];
        eb.ldc = K;
        eb.Aout = s->dZ[i];
        eb.lda_out = K;
        eb.AoutT = s->DT[i];
        eb.ldT = LT;
        eb.dbias = s->g + kL.b[l - 1];
        return gemm<EPI_DSILU>(D, N, s->wbfT + kL.w[l], N, R, K, N, eb, s->tc_err, st);
    };
    const int ygrid = (int)std::min<int64_t>(rows, 512);
    // output layer
    int cur = 0;
    {
        const int l = kLayers - 1, N = out_dim(l);
        if (e == cudaSuccess)
            e = weight_grad(s->OT, l);
        if (e == cudaSuccess) {
            colsum_kernel<<<dim3((N + 127) / 128, ygrid), 128, 0, st>>>(s->dOut, rows, N,
                                                                        s->g + kL.b[l]);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = input_grad(s->dOut, l, cur);
    }
    // hidden layers: dZ[cur] / DT[cur] hold layer l's output gradient
    for (int l = kLayers - 2; l >= 0 && e == cudaSuccess; --l) {
        e = weight_grad(s->DT[cur], l);
        if (l > 0 && e == cudaSuccess)
            e = input_grad(s->dZ[cur], l, cur ^ 1);
        cur ^= 1;
    }
    return e;
}

static int check_rows(int64_t n)
{
    if (n < 0 || n > (int64_t)1 << 30)
        return fail(KERR_EINVAL, "surrogate: row count out of range");
    return KERR_OK;
}

// Inference forward: the fused tensor-core kernel (kerr_mlp_tc.cu) on the
// current bf16 weights, packed into its operand layout first.
static int forward_fused(kerr_surrogate *s, const float *in, int64_t n, float *out,
                         cudaStream_t st)
{
    SURR_CUDA(pack_weights(s->wbf, kL.w, s->wpk, st));
    const float *bias[kLayers];
    for (int l = 0; l < kLayers; ++l)
        bias[l] = s->w + kL.b[l];
    SURR_CUDA(forward_tc(in, n, out, s->wpk, bias, s->tc_err, s->sms, st));
    return KERR_OK;
}

// After a synchronisation: KERR_ECUDA if a fused-forward pipeline wait gave up.
static int check_tc(kerr_surrogate *s)
{
    unsigned h = 0;
    SURR_CUDA(cudaMemcpy(&h, s->tc_err, sizeof h, cudaMemcpyDeviceToHost));
    if (h) {
        cudaMemset(s->tc_err, 0, sizeof h);
        return fail(KERR_ECUDA, "surrogate: tensor-core pipeline wait timed out");
    }
    return KERR_OK;
}

// The same forward on the layer-by-layer GEMM kernels (training path).
static int forward_gemm(kerr_surrogate *s, const float *in, int64_t n, float *out,
                        cudaStream_t st)
{
    const int64_t chunk = 1 << 20;
    int rc = ensure_batch(s, std::min(n, chunk), false);
    if (rc)
        return rc;
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t rows = std::min(chunk, n - r0);
        input_kernel<<<grid_1d(rows * kInPad), 256, 0, st>>>(in + r0 * kIn, s->A[0], rows);
        SURR_CUDA(cudaGetLastError());
        SURR_CUDA(forward_rows(s, rows, false, st));
        SURR_CUDA(cudaMemcpy2DAsync(out + r0 * kOut, kOut * sizeof(float), s->out,
                                    kOutPad * sizeof(float), kOut * sizeof(float), rows,
                                    cudaMemcpyDeviceToDevice, st));
    }
    return KERR_OK;
}

extern "C" int kerr_surrogate_forward(kerr_surrogate *s, const float *in, int64_t n, float *out,
                                      void *stream)
{
    return kerr_surrogate_forward_impl(s, in, n, out, KERR_SURR_FWD_TENSOR_CORE, stream);
}

extern "C" int kerr_surrogate_forward_impl(kerr_surrogate *s, const float *in, int64_t n,
                                           float *out, int32_t impl, void *stream)
{
    if (!s || (n > 0 && (!in || !out)))
        return fail(KERR_EINVAL, "kerr_surrogate_forward: NULL argument");
    if (impl != KERR_SURR_FWD_TENSOR_CORE && impl != KERR_SURR_FWD_GEMM)
        return fail(KERR_EINVAL, "kerr_surrogate_forward: unknown implementation");
    int rc = check_rows(n);
    if (rc || n == 0)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (impl == KERR_SURR_FWD_GEMM) {
        rc = forward_gemm(s, in, n, out, st);
        if (rc)
            return rc;
        SURR_CUDA(cudaStreamSynchronize(st));
        return check_tc(s);
    }
    rc = forward_fused(s, in, n, out, st);
    if (rc)
        return rc;
    SURR_CUDA(cudaStreamSynchronize(st));
    return check_tc(s);
}

// The packed training weights, refreshed from the bf16 copy when the GEMM
// path's Adam was the last to change the weights.
static cudaError_t ensure_packed(kerr_surrogate *s, cudaStream_t st)
{
    if (s->wtp_valid)
        return cudaSuccess;
    const cudaError_t e = train_pack(s->wbf, kL.w, s->wtp, st);
    if (e == cudaSuccess)
        s->wtp_valid = true;
    return e;
}

// The transposed bf16 weights of the GEMM path's input gradients, refreshed
// from the bf16 copy after fused Adam steps.
static cudaError_t ensure_wbfT(kerr_surrogate *s, cudaStream_t st)
{
    if (s->wbfT_valid)
        return cudaSuccess;
    transpose_weights_kernel<<<grid_1d(kL.total), 256, 0, st>>>(s->wbf, s->wbfT, woffsets());
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        s->wbfT_valid = true;
    return e;
}

static void train_biases(const kerr_surrogate *s, const float *bias[kLayers])
{
    for (int l = 0; l < kLayers; ++l)
        bias[l] = s->w + kL.b[l];
}

extern "C" int kerr_surrogate_grad_impl(kerr_surrogate *s, const float *in,
                                        const float *targets, const float *mask, int64_t n,
                                        float *loss, int32_t impl, void *stream)
{
    if (!s || !in || !targets || !mask || n < 1)
        return fail(KERR_EINVAL, "kerr_surrogate_grad: bad argument");
    if (impl != KERR_SURR_TRAIN_FUSED && impl != KERR_SURR_TRAIN_GEMM)
        return fail(KERR_EINVAL, "kerr_surrogate_grad: unknown implementation");
    int rc = check_rows(n);
    if (rc)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (impl == KERR_SURR_TRAIN_FUSED) {
        rc = ensure_train(s, n);
        if (rc)
            return rc;
        const float *bias[kLayers];
        train_biases(s, bias);
        SURR_CUDA(ensure_packed(s, st));
        SURR_CUDA(cudaMemsetAsync(s->loss, 0, sizeof(float), st));
        SURR_CUDA(train_chain(in, targets, mask, n, nullptr, s->loss, bias, s->wtp, s->tb,
                              s->tc_err, s->sms, st));
        SURR_CUDA(train_grads(s->tb, n, s->part, kL.total, kL.w, kL.b, s->tc_err, s->sms, st));
        SURR_CUDA(train_reduce(s->part, train_splits(n, s->sms), kL.total, s->g, st));
    } else {
        rc = ensure_batch(s, n, true);
        if (rc)
            return rc;
        SURR_CUDA(ensure_wbfT(s, st));
        input_kernel<<<grid_1d(n * kInPad), 256, 0, st>>>(in, s->A[0], n, s->AT[0], s->ldT);
        SURR_CUDA(cudaGetLastError());
        SURR_CUDA(forward_rows(s, n, true, st));
        SURR_CUDA(cudaMemsetAsync(s->loss, 0, sizeof(float), st));
        loss_kernel<<<grid_1d(n, 64), 64, 0, st>>>(s->out, targets, mask, n, 1.0f / (float)n,
                                                   s->dOut, s->loss, s->OT, s->ldT);
        SURR_CUDA(cudaGetLastError());
        SURR_CUDA(backward_rows(s, n, st));
    }
    float h = 0.f;
    SURR_CUDA(cudaMemcpyAsync(&h, s->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    SURR_CUDA(cudaStreamSynchronize(st));
    rc = check_tc(s);
    if (rc)
        return rc;
    if (loss)
        *loss = h;
    return KERR_OK;
}

extern "C" int kerr_surrogate_grad(kerr_surrogate *s, const float *in, const float *targets,
                                   const float *mask, int64_t n, float *loss, void *stream)
{
    return kerr_surrogate_grad_impl(s, in, targets, mask, n, loss, KERR_SURR_TRAIN_FUSED,
                                    stream);
}

extern "C" int kerr_surrogate_train_impl(kerr_surrogate *s, const float *in,
                                         const float *targets, const float *mask, int64_t n,
                                         int32_t epochs, int32_t batch, float lr,
                                         float *loss_per_epoch, int32_t impl, void *stream)
{
    if (!s || !in || !targets || !mask || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.f))
        return fail(KERR_EINVAL, "kerr_surrogate_train: bad argument");
    if (impl != KERR_SURR_TRAIN_FUSED && impl != KERR_SURR_TRAIN_GEMM)
        return fail(KERR_EINVAL, "kerr_surrogate_train: unknown implementation");
    int rc = check_rows(n);
    if (rc)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t B = std::min<int64_t>(batch, n);
    const bool fused = impl == KERR_SURR_TRAIN_FUSED;
    rc = fused ? ensure_train(s, B) : ensure_batch(s, B, true);
    if (rc)
        return rc;
    const float *bias[kLayers];
    train_biases(s, bias);
    const int64_t steps_per_epoch = n / B;
    const int64_t total = std::max<int64_t>(1, steps_per_epoch * epochs);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    // One training step = one fixed sequence of launches whose per-step values
    // (batch rows, epoch, learning rate, bias corrections) are computed on the
    // device: it is captured once as a CUDA graph of U steps and replayed, on
    // a private stream ordered after the caller's.
    float *d_epoch = nullptr;
    StepCtl *ctl = nullptr;
    float3 *sched = nullptr;
    // cosine learning-rate schedule from lr down to 0.05 lr over the run, and
    // Adam's bias corrections 1 / (1 - beta^t) at t = step0 + k + 1
    std::vector<float3> hs((size_t)total);
    for (int64_t k = 0; k < total; ++k) {
        const double frac = (double)k / (double)total;
        const double t = (double)(s->step + k + 1);
        hs[k] = make_float3((float)(lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(M_PI * frac)))),
                            (float)(1.0 / (1.0 - std::pow((double)b1, t))),
                            (float)(1.0 / (1.0 - std::pow((double)b2, t))));
    }
    cudaStream_t cs = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraph_t gU = nullptr, g1 = nullptr;
    cudaGraphExec_t xU = nullptr, x1 = nullptr;
    auto enqueue_step = [&](cudaStream_t q) -> cudaError_t {
        train_step_kernel<<<1, 32, 0, q>>>(ctl, sched, steps_per_epoch, B);
        if (fused) {
            // chain, partial gradients, Adam on their sum
            cudaError_t e = train_chain(in, targets, mask, B, ctl, d_epoch, bias, s->wtp, s->tb,
                                        s->tc_err, s->sms, q);
            if (e == cudaSuccess)
                e = train_grads(s->tb, B, s->part, kL.total, kL.w, kL.b, s->tc_err, s->sms, q);
            if (e == cudaSuccess)
                e = train_adam(s->w, s->part, train_splits(B, s->sms), s->m, s->v, s->wbf,
                               s->wtp, kL.w, kL.total, ctl, b1, b2, eps, q);
            return e;
        }
        input_kernel<<<grid_1d(B * kInPad), 256, 0, q>>>(in, s->A[0], B, s->AT[0], s->ldT, ctl);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = forward_rows(s, B, true, q);
        if (e == cudaSuccess) {
            loss_kernel<<<grid_1d(B, 64), 64, 0, q>>>(s->out, targets, mask, B, 1.0f / (float)B,
                                                      s->dOut, d_epoch, s->OT, s->ldT, ctl);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = backward_rows(s, B, q);
        if (e == cudaSuccess) {
            adam_kernel<<<grid_1d(kL.total), 256, 0, q>>>(s->w, s->g, s->m, s->v, s->wbf, s->wbfT,
                                                          woffsets(), kL.total, ctl, b1, b2, eps);
            e = cudaGetLastError();
        }
        return e;
    };
    auto capture = [&](int steps, cudaGraph_t *g, cudaGraphExec_t *x) -> cudaError_t {
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (int u = 0; u < steps && e == cudaSuccess; ++u)
            e = enqueue_step(cs);
        cudaGraph_t gg = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &gg);
        if (e == cudaSuccess)
            e = e2;
        *g = gg;
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(x, gg, 0);
        return e;
    };
    const int U = (int)std::min<int64_t>(8, total);
    cudaError_t e = dev_alloc(&d_epoch, sizeof(float) * epochs);
    if (e == cudaSuccess)
        e = dev_alloc(&ctl, sizeof(StepCtl));
    if (e == cudaSuccess)
        e = dev_alloc(&sched, sizeof(float3) * (size_t)total);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sched, hs.data(), sizeof(float3) * (size_t)total,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&ev1, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_epoch, 0, sizeof(float) * epochs, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctl, 0, sizeof(StepCtl), st);
    if (e == cudaSuccess)
        e = fused ? ensure_packed(s, st) : ensure_wbfT(s, st);
    if (e == cudaSuccess)
        e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(cs, ev0, 0);
    if (e == cudaSuccess)
        e = capture(U, &gU, &xU);
    if (e == cudaSuccess && total % U)
        e = capture(1, &g1, &x1);
    for (int64_t i = 0; i < total / U && e == cudaSuccess; ++i)
        e = cudaGraphLaunch(xU, cs);
    for (int64_t i = 0; i < total % U && e == cudaSuccess; ++i)
        e = cudaGraphLaunch(x1, cs);
    if (e == cudaSuccess)
        e = cudaEventRecord(ev1, cs);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(st, ev1, 0);
    std::vector<float> h(epochs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d_epoch, sizeof(float) * epochs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        s->step += total;
    if (!fused)
        s->wtp_valid = false;       // the GEMM path's Adam leaves the packed weights stale
    else
        s->wbfT_valid = false;      // the fused Adam leaves the transposed copy stale
    if (xU)
        cudaGraphExecDestroy(xU);
    if (x1)
        cudaGraphExecDestroy(x1);
    if (gU)
        cudaGraphDestroy(gU);
    if (g1)
        cudaGraphDestroy(g1);
    if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
    }
    if (ev0)
        cudaEventDestroy(ev0);
    if (ev1)
        cudaEventDestroy(ev1);
    cudaFree(d_epoch);
    cudaFree(ctl);
    cudaFree(sched);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ECUDA, "kerr_surrogate_train: launch failed");
    }
    rc = check_tc(s);
    if (rc)
        return rc;
    if (loss_per_epoch)
        for (int ep = 0; ep < epochs; ++ep)
            loss_per_epoch[ep] = h[ep] / (float)std::max<int64_t>(1, steps_per_epoch);
    return KERR_OK;
}

extern "C" int kerr_surrogate_train(kerr_surrogate *s, const float *in, const float *targets,
                                    const float *mask, int64_t n, int32_t epochs, int32_t batch,
                                    float lr, float *loss_per_epoch, void *stream)
{
    return kerr_surrogate_train_impl(s, in, targets, mask, n, epochs, batch, lr, loss_per_epoch,
                                     KERR_SURR_TRAIN_FUSED, stream);
}

// ===========================================================================
// training targets from integrated rays
// ===========================================================================
namespace {

__global__ void targets_kernel(const double *__restrict__ pts, const int32_t *__restrict__ status,
                               const float *__restrict__ cross, int64_t n, float *__restrict__ in,
                               float *__restrict__ tgt, float *__restrict__ msk)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double *p = pts + 4 * i;
        in[4 * i + 0] = (float)p[0] / KERR_SURR_INPUT_SCALE;
        in[4 * i + 1] = (float)p[1] / KERR_SURR_INPUT_SCALE;
        in[4 * i + 2] = (float)p[2];
        in[4 * i + 3] = (float)cos(p[3]);
        float *y = tgt + kOut * i;
        float *m = msk + kOut * i;
        y[0] = status[i] == ST_CAPTURED ? 1.0f : 0.0f;
        m[0] = 1.0f;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float r = cross[(2 * c) * n + i], ph = cross[(2 * c + 1) * n + i];
            const bool ok = !isnan(r) && !isnan(ph);
            y[1 + 3 * c] = ok ? 0.5f * (logf(r) - 2.0f) : 0.0f;
            y[2 + 3 * c] = ok ? cosf(ph) : 0.0f;
            y[3 + 3 * c] = ok ? sinf(ph) : 0.0f;
            m[1 + 3 * c] = m[2 + 3 * c] = m[3 + 3 * c] = ok ? 1.0f : 0.0f;
        }
        const float g = cross[4 * n + i];
        y[7] = isnan(g) ? 0.0f : g - 1.0f;
        m[7] = isnan(g) ? 0.0f : 1.0f;
    }
}

} // namespace

extern "C" int kerr_surrogate_targets(kerr_ctx *ctx, const double *points, int64_t n, double r_obs,
                                      const kerr_opts *opts, float *in, float *targets,
                                      float *mask, void *stream)
{
    if (!ctx || !points || !in || !targets || !mask || n < 1)
        return fail(KERR_EINVAL, "kerr_surrogate_targets: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    double *x = nullptr, *k = nullptr;
    int32_t *stat = nullptr, *nst = nullptr;
    float *cr = nullptr;
    cudaError_t e = dev_alloc(&x, (size_t)n * 4 * sizeof(double));
    if (e == cudaSuccess)
        e = dev_alloc(&k, (size_t)n * 4 * sizeof(double));
    if (e == cudaSuccess)
        e = dev_alloc(&stat, (size_t)n * sizeof(int32_t));
    if (e == cudaSuccess)
        e = dev_alloc(&nst, (size_t)n * sizeof(int32_t));
    if (e == cudaSuccess)
        e = dev_alloc(&cr, (size_t)n * 5 * sizeof(float));
    int rc = KERR_OK;
    if (e != cudaSuccess) {
        cudaGetLastError();
        rc = fail(KERR_ENOMEM, "kerr_surrogate_targets: allocation");
    }
    if (rc == KERR_OK)
        rc = kerr_trace_points(ctx, points, n, r_obs, opts, x, k, stat, nst, nullptr, cr, stream);
    if (rc == KERR_OK) {
        targets_kernel<<<grid_1d(n), 256, 0, st>>>(points, stat, cr, n, in, targets, mask);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(KERR_ECUDA, "kerr_surrogate_targets: kernel failed");
        }
    }
    cudaStreamSynchronize(st);
    cudaFree(x);
    cudaFree(k);
    cudaFree(stat);
    cudaFree(nst);
    cudaFree(cr);
    return rc;
}

// ===========================================================================
// rendering with integrator fallback
// ===========================================================================
namespace {

// Bardeen's critical curve of a distant observer (M = 1): spherical photon
// orbits r in [r_ph+, r_ph-] with xi(r) = -(r^3 - 3r^2 + a^2 r + a^2)/(a(r-1)),
// eta(r) = -r^3 (r^3 - 6r^2 + 9r - 4a^2)/(a^2 (r-1)^2), seen at
// alpha = -xi / sin i, beta = +-sqrt(eta + a^2 cos^2 i - xi^2 cot^2 i).  The
// camera's alpha axis is (0, 1, 0) with n = (sin i, 0, cos i), so its alpha
// is Bardeen's alpha.  For a -> 0 the curve is the circle of radius 3 sqrt 3.
__device__ __forceinline__ double crit_beta2(double a, double si, double ci, double r,
                                             double &alpha)
{
    const double xi = -(r * r * r - 3.0 * r * r + a * a * r + a * a) / (a * (r - 1.0));
    const double eta =
        -r * r * r * (r * r * r - 6.0 * r * r + 9.0 * r - 4.0 * a * a) / (a * a * (r - 1.0) * (r - 1.0));
    alpha = -xi / si;
    return eta + a * a * ci * ci - xi * xi * (ci * ci) / (si * si);
}

// The visible part of the curve is the r interval where beta^2 >= 0: one
// block samples beta^2 over [r_p, r_r], keeps the first and last
// non-negative samples and bisects each edge to double precision.
__global__ void crit_interval_kernel(double a, double incl, double *__restrict__ rr_out)
{
    constexpr int S = 4096;
    __shared__ int lo_i, hi_i;
    const double si = sin(incl), ci = cos(incl);
    const double rp = 2.0 * (1.0 + cos(2.0 / 3.0 * acos(-fabs(a))));
    const double rr = 2.0 * (1.0 + cos(2.0 / 3.0 * acos(fabs(a))));
    if (threadIdx.x == 0) {
        lo_i = S;
        hi_i = -1;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < S; j += blockDim.x) {
        double al;
        const double r = rp + (rr - rp) * (j + 0.5) / S;
        if (crit_beta2(a, si, ci, r, al) >= 0.0) {
            atomicMin(&lo_i, j);
            atomicMax(&hi_i, j);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r1 = NAN, r2 = NAN;
        if (hi_i >= lo_i) {
            // lower edge: beta^2 < 0 at rA, >= 0 at rB
            double rA = rp + (rr - rp) * (lo_i - 0.5) / S, rB = rp + (rr - rp) * (lo_i + 0.5) / S;
            rA = fmax(rA, rp);
            double al;
            if (crit_beta2(a, si, ci, rA, al) >= 0.0)
                rB = rA;
            for (int it = 0; it < 60; ++it) {
                const double rm = 0.5 * (rA + rB);
                if (crit_beta2(a, si, ci, rm, al) >= 0.0)
                    rB = rm;
                else
                    rA = rm;
            }
            r1 = rB;
            double rC = rp + (rr - rp) * (hi_i + 0.5) / S, rD = rp + (rr - rp) * (hi_i + 1.5) / S;
            rD = fmin(rD, rr);
            if (crit_beta2(a, si, ci, rD, al) >= 0.0)
                rC = rD;
            for (int it = 0; it < 60; ++it) {
                const double rm = 0.5 * (rC + rD);
                if (crit_beta2(a, si, ci, rm, al) >= 0.0)
                    rC = rm;
                else
                    rD = rm;
            }
            r2 = rC;
        }
        rr_out[0] = r1;
        rr_out[1] = r2;
    }
}

// Samples of the curve, `ns` per branch (2 ns points; NaN if none visible),
// cosine-spaced in r over the visible interval (dense at the ends, where
// beta goes to zero like the square root of the distance in r).
__global__ void crit_curve_kernel(double a, double incl, int ns, const double *__restrict__ rr,
                                  float2 *__restrict__ pts)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns)
        return;
    const double si = sin(incl), ci = cos(incl);
    const float nanf_ = __int_as_float(0x7fc00000);
    float2 p0 = make_float2(nanf_, nanf_);
    float2 p1 = p0;
    if (fabs(a) < 1e-4) {
        const double b = 3.0 * sqrt(3.0);
        const double th = 2.0 * M_PI * (j + 0.5) / ns;
        const double th2 = th + M_PI / ns;
        p0 = make_float2((float)(b * cos(th)), (float)(b * sin(th)));
        p1 = make_float2((float)(b * cos(th2)), (float)(b * sin(th2)));
    } else if (!isnan(rr[0])) {
        const double u = 0.5 * (1.0 - cos(M_PI * j / (ns - 1)));
        const double r = rr[0] + (rr[1] - rr[0]) * u;
        double al;
        const double b2 = fmax(0.0, crit_beta2(a, si, ci, r, al));
        const double be = sqrt(b2);
        p0 = make_float2((float)al, (float)be);
        p1 = make_float2((float)al, (float)-be);
    }
    pts[j] = p0;
    pts[ns + j] = p1;
}

// Annulus holding the curve samples: centre (bounding-box midpoint of the
// finite samples) and the smallest / largest sample distance from it.  A
// pixel at distance d from the centre is at least min over samples of
// |d - |q - c|| from every sample (triangle inequality), so with d outside
// [rmin - crit, rmax + crit] no sample is within crit.  One block.
__global__ void curve_bounds_kernel(const float2 *__restrict__ curve, int ncurve,
                                    float4 *__restrict__ bounds)
{
    __shared__ float red[4][256];
    float x0 = 3.0e38f, x1 = -3.0e38f, y0 = 3.0e38f, y1 = -3.0e38f;
    for (int j = threadIdx.x; j < ncurve; j += blockDim.x) {
        const float2 q = curve[j];
        if (isfinite(q.x) && isfinite(q.y)) {
            x0 = fminf(x0, q.x);
            x1 = fmaxf(x1, q.x);
            y0 = fminf(y0, q.y);
            y1 = fmaxf(y1, q.y);
        }
    }
    red[0][threadIdx.x] = x0;
    red[1][threadIdx.x] = -x1;
    red[2][threadIdx.x] = y0;
    red[3][threadIdx.x] = -y1;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 4; ++k)
                red[k][threadIdx.x] = fminf(red[k][threadIdx.x], red[k][threadIdx.x + w]);
        __syncthreads();
    }
    const float cx = 0.5f * (red[0][0] - red[1][0]), cy = 0.5f * (red[2][0] - red[3][0]);
    __syncthreads();
    float r0 = 3.0e38f, r1 = -3.0e38f;
    for (int j = threadIdx.x; j < ncurve; j += blockDim.x) {
        const float2 q = curve[j];
        if (isfinite(q.x) && isfinite(q.y)) {
            const float d = hypotf(q.x - cx, q.y - cy);
            r0 = fminf(r0, d);
            r1 = fmaxf(r1, d);
        }
    }
    red[0][threadIdx.x] = r0;
    red[1][threadIdx.x] = -r1;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 2; ++k)
                red[k][threadIdx.x] = fminf(red[k][threadIdx.x], red[k][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *bounds = make_float4(cx, cy, red[0][0], -red[1][0]);   // no sample: rmin > rmax
}

// Gate and decode: one pass over the pixels.  Network outputs o [n][8];
// fallback when p in [p_lo, p_hi] or distance to the curve < crit_dist
// (the sample scan only for pixels inside the annulus of curve_bounds_kernel
// widened by crit_dist); fallback pixels are appended (warp-aggregated) to
// idx.
__global__ void __launch_bounds__(256) gate_kernel(const float *__restrict__ o, kerr_camera cam,
                                                   const float2 *__restrict__ curve, int ncurve,
                                                   const float4 *__restrict__ bounds,
                                                   float p_lo, float p_hi, float crit_dist,
                                                   int64_t n, float *__restrict__ out,
                                                   uint8_t *__restrict__ fb,
                                                   int64_t *__restrict__ idx,
                                                   unsigned long long *__restrict__ count)
{
    extern __shared__ float2 sc[];
    for (int j = threadIdx.x; j < ncurve; j += blockDim.x)
        sc[j] = curve[j];
    const float4 bd = *bounds;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        bool use_fb = false;
        if (i < n) {
            const float *oi = o + kOut * i;
            const float p = 1.0f / (1.0f + __expf(-oi[0]));
            const int64_t px = i % cam.nx, qy = i / cam.nx;
            const float al = (float)(-cam.half_width + (px + 0.5) * 2.0 * cam.half_width / cam.nx);
            const float be = (float)(-cam.half_width + (qy + 0.5) * 2.0 * cam.half_width / cam.ny);
            float d2 = 3.0e38f;
            const float dc = hypotf(al - bd.x, be - bd.y);
            if (dc >= bd.z - crit_dist && dc <= bd.w + crit_dist) {
                for (int j = 0; j < ncurve; ++j) {
                    const float dx = sc[j].x - al, dy = sc[j].y - be;
                    const float dd = dx * dx + dy * dy;
                    d2 = dd < d2 ? dd : d2;      // NaN samples never win
                }
            }
            use_fb = (p >= p_lo && p <= p_hi) || d2 < crit_dist * crit_dist;
            const float nan = __int_as_float(0x7fc00000);
            out[i] = p;
            const bool cap = p >= 0.5f;
            for (int c = 0; c < 2; ++c) {
                const float lr = oi[1 + 3 * c], cph = oi[2 + 3 * c], sph = oi[3 + 3 * c];
                out[(1 + 2 * c) * n + i] = cap ? nan : __expf(2.0f * lr + 2.0f);
                out[(2 + 2 * c) * n + i] = cap ? nan : atan2f(sph, cph);
            }
            out[5 * n + i] = cap ? nan : oi[7] + 1.0f;
            if (fb)
                fb[i] = use_fb ? 1 : 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, use_fb);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long b = 0;
            if (lane == leader)
                b = atomicAdd(count, (unsigned long long)__popc(m));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (use_fb)
                idx[b + __popc(m & ((1u << lane) - 1u))] = i;
        }
    }
}

// Network inputs (alpha/s, beta/s, a, cos i) of every pixel of a camera.
__global__ void surr_query_kernel(float *in, kerr_camera cam, int64_t n)
{
    const float ci = (float)cos(cam.incl);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t px = i % cam.nx, qy = i / cam.nx;
        const double al = -cam.half_width + (px + 0.5) * 2.0 * cam.half_width / cam.nx;
        const double be = -cam.half_width + (qy + 0.5) * 2.0 * cam.half_width / cam.ny;
        in[4 * i + 0] = (float)al / KERR_SURR_INPUT_SCALE;
        in[4 * i + 1] = (float)be / KERR_SURR_INPUT_SCALE;
        in[4 * i + 2] = (float)cam.a;
        in[4 * i + 3] = ci;
    }
}

// Scatter the integrator's results of the fallback pixels into the planes.
__global__ void merge_kernel(const int64_t *__restrict__ idx,
                             const unsigned long long *__restrict__ count,
                             const int32_t *__restrict__ status, const float *__restrict__ cross,
                             int64_t cap_rows, int64_t n, float *__restrict__ out)
{
    const int64_t live = (int64_t)*count;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < live;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx[j];
        out[i] = status[j] == ST_CAPTURED ? 1.0f : 0.0f;
        for (int c = 0; c < 5; ++c)
            out[(1 + c) * n + i] = cross[c * cap_rows + j];
    }
}

} // namespace

static int ensure_render(RenderScratch &r, int64_t n, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (!r.curve) {
        e = dev_alloc(&r.curve, (size_t)2 * kCurveSamples * sizeof(float2));
        if (e == cudaSuccess)
            e = dev_alloc(&r.rint, 2 * sizeof(double));
        if (e == cudaSuccess)
            e = dev_alloc(&r.bounds, sizeof(float4));
        if (e == cudaSuccess)
            e = dev_alloc(&r.cnt, sizeof(unsigned long long));
    }
    if (e == cudaSuccess && n > r.cap_n) {
        cudaStreamSynchronize(st);
        cudaFree(r.in);
        cudaFree(r.o);
        cudaFree(r.idx);
        r.in = r.o = nullptr;
        r.idx = nullptr;
        r.cap_n = 0;
        e = dev_alloc(&r.in, (size_t)n * kIn * sizeof(float));
        if (e == cudaSuccess)
            e = dev_alloc(&r.o, (size_t)n * kOut * sizeof(float));
        if (e == cudaSuccess)
            e = dev_alloc(&r.idx, (size_t)n * sizeof(int64_t));
        if (e == cudaSuccess)
            r.cap_n = n;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_render(r);
        return fail(KERR_ENOMEM, "kerr_surrogate_render: scratch allocation");
    }
    return KERR_OK;
}

static int ensure_fallback(RenderScratch &r, int64_t m, cudaStream_t st)
{
    if (m <= r.cap_m)
        return KERR_OK;
    cudaStreamSynchronize(st);
    cudaFree(r.x);
    cudaFree(r.k);
    cudaFree(r.stat);
    cudaFree(r.nst);
    cudaFree(r.crs);
    r.x = r.k = nullptr;
    r.stat = r.nst = nullptr;
    r.crs = nullptr;
    r.cap_m = 0;
    const int64_t want = std::max<int64_t>(m, 1 << 16);
    cudaError_t e = dev_alloc(&r.x, (size_t)want * 4 * sizeof(double));
    if (e == cudaSuccess)
        e = dev_alloc(&r.k, (size_t)want * 4 * sizeof(double));
    if (e == cudaSuccess)
        e = dev_alloc(&r.stat, (size_t)want * sizeof(int32_t));
    if (e == cudaSuccess)
        e = dev_alloc(&r.nst, (size_t)want * sizeof(int32_t));
    if (e == cudaSuccess)
        e = dev_alloc(&r.crs, (size_t)want * 5 * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_render(r);
        return fail(KERR_ENOMEM, "kerr_surrogate_render: fallback buffers");
    }
    r.cap_m = want;
    return KERR_OK;
}

extern "C" int kerr_surrogate_render(kerr_ctx *ctx, kerr_surrogate *s, const kerr_camera *cam,
                                     const kerr_opts *opts, float p_lo, float p_hi,
                                     float crit_dist, float *out, uint8_t *fallback,
                                     int64_t *n_fallback, void *stream)
{
    if (!ctx || !s || !cam || !opts || !out)
        return fail(KERR_EINVAL, "kerr_surrogate_render: NULL argument");
    if (cam->nx <= 0 || cam->ny <= 0 || !(std::fabs(cam->a) <= 1.0))
        return fail(KERR_EINVAL, "kerr_surrogate_render: invalid camera");
    const int64_t n = (int64_t)cam->nx * cam->ny;
    cudaStream_t st = (cudaStream_t)stream;
    RenderScratch &r = *s->render;
    int rc = ensure_render(r, n, st);
    if (rc)
        return rc;
    const int ns = kCurveSamples;
    unsigned long long hcount = 0;
    // network inputs from the pixel grid, then the fused forward
    cudaError_t e = cudaMemsetAsync(r.cnt, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        surr_query_kernel<<<grid_1d(n), 256, 0, st>>>(r.in, *cam, n);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ECUDA, "kerr_surrogate_render: query kernel");
    }
    rc = forward_fused(s, r.in, n, r.o, st);
    if (rc)
        return rc;
    // critical curve, gate + decode, compaction of the fallback pixels
    if (std::fabs(cam->a) >= 1e-4)
        crit_interval_kernel<<<1, 256, 0, st>>>(cam->a, cam->incl, r.rint);
    crit_curve_kernel<<<(ns + 127) / 128, 128, 0, st>>>(cam->a, cam->incl, ns, r.rint, r.curve);
    curve_bounds_kernel<<<1, 256, 0, st>>>(r.curve, 2 * ns, r.bounds);
    gate_kernel<<<grid_1d(n), 256, 2 * ns * sizeof(float2), st>>>(
        r.o, *cam, r.curve, 2 * ns, r.bounds, p_lo, p_hi, crit_dist, n, out, fallback, r.idx,
        r.cnt);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hcount, r.cnt, sizeof hcount, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KERR_ECUDA, "kerr_surrogate_render: gate");
    }
    rc = check_tc(s);
    if (rc)
        return rc;
    // the integrator on the fallback pixels, merged into the planes
    if (hcount > 0) {
        const int64_t m = (int64_t)hcount;
        rc = ensure_fallback(r, m, st);
        // capacity = the buffers' size (the live count is read on the device),
        // so that renders of any fallback count replay one captured graph
        if (rc == KERR_OK)
            rc = kerr_trace_camera_list(ctx, cam, r.idx, r.cnt, r.cap_m, opts, r.x, r.k, r.stat,
                                        r.nst, nullptr, r.crs, stream);
        if (rc == KERR_OK) {
            merge_kernel<<<grid_1d(m), 256, 0, st>>>(r.idx, r.cnt, r.stat, r.crs, r.cap_m, n,
                                                     out);
            if (cudaGetLastError() != cudaSuccess) {
                cudaGetLastError();
                rc = fail(KERR_ECUDA, "kerr_surrogate_render: merge");
            }
        }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == KERR_OK) {
        cudaGetLastError();
        rc = fail(KERR_ECUDA, "kerr_surrogate_render: synchronisation");
    }
    if (n_fallback)
        *n_fallback = (int64_t)hcount;
    return rc;
}


// ---------------------------------------------------------------------------
// Parameter files: a 96-byte header and the FP32 parameter vector, both
// little-endian (the byte order of every host this library builds for).
// Host code only; the checksum is FNV-1a over the parameter bytes.
// ---------------------------------------------------------------------------
namespace {

struct ParamFileHeader {
    char magic[8];          // "KERRSURR"
    uint32_t version;       // 1
    uint32_t header_bytes;  // 96
    int64_t num_params;
    int32_t layers;
    int32_t in_width[kLayers];
    int32_t out_width[kLayers];
    int32_t live_in, live_out;
    float input_scale;
    uint32_t checksum;
    uint8_t reserved[12];
};
static_assert(sizeof(ParamFileHeader) == 96, "parameter file header layout");

const char kParamMagic[8] = {'K', 'E', 'R', 'R', 'S', 'U', 'R', 'R'};

uint32_t fnv1a(const void *data, size_t bytes)
{
    const unsigned char *p = static_cast<const unsigned char *>(data);
    uint32_t h = 2166136261u;
    for (size_t i = 0; i < bytes; ++i) {
        h ^= p[i];
        h *= 16777619u;
    }
    return h;
}

ParamFileHeader expected_header()
{
    ParamFileHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kParamMagic, sizeof h.magic);
    h.version = 1;
    h.header_bytes = sizeof(ParamFileHeader);
    h.num_params = (int64_t)kL.total;
    h.layers = kLayers;
    for (int l = 0; l < kLayers; ++l) {
        h.in_width[l] = in_dim(l);
        h.out_width[l] = out_dim(l);
    }
    h.live_in = kIn;
    h.live_out = kOut;
    h.input_scale = KERR_SURR_INPUT_SCALE;
    return h;
}

} // namespace

extern "C" int kerr_params_write(const char *path, const float *params, int64_t n)
{
    if (!path || !params)
        return fail(KERR_EINVAL, "kerr_params_write: NULL argument");
    if (n != (int64_t)kL.total)
        return fail(KERR_EINVAL, "kerr_params_write: n is not kerr_surrogate_num_params()");
    ParamFileHeader h = expected_header();
    const size_t bytes = (size_t)n * sizeof(float);
    h.checksum = fnv1a(params, bytes);
    FILE *f = std::fopen(path, "wb");
    if (!f)
        return fail(KERR_EINVAL, "kerr_params_write: cannot open the file for writing");
    const bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 &&
                    std::fwrite(params, 1, bytes, f) == bytes;
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed)
        return fail(KERR_EINVAL, "kerr_params_write: write failed");
    return KERR_OK;
}

extern "C" int kerr_params_read(const char *path, float *params, int64_t n)
{
    if (!path || !params)
        return fail(KERR_EINVAL, "kerr_params_read: NULL argument");
    if (n != (int64_t)kL.total)
        return fail(KERR_EINVAL, "kerr_params_read: n is not kerr_surrogate_num_params()");
    FILE *f = std::fopen(path, "rb");
    if (!f)
        return fail(KERR_EINVAL, "kerr_params_read: cannot open the file");
    ParamFileHeader h;
    const size_t bytes = (size_t)n * sizeof(float);
    bool ok = std::fread(&h, sizeof h, 1, f) == 1;
    const ParamFileHeader want = expected_header();
    // every field but the checksum must be this network's
    ParamFileHeader cmp = h;
    if (ok)
        cmp.checksum = 0;
    if (!ok || std::memcmp(&cmp, &want, sizeof want) != 0) {
        std::fclose(f);
        return fail(KERR_EINVAL, "kerr_params_read: not a parameter file of this network "
                                 "(magic, version or layer widths differ)");
    }
    ok = std::fread(params, 1, bytes, f) == bytes;
    const bool extra = ok && std::fgetc(f) != EOF;
    std::fclose(f);
    if (!ok || extra)
        return fail(KERR_EINVAL, "kerr_params_read: the file has the wrong length");
    if (fnv1a(params, bytes) != h.checksum)
        return fail(KERR_EINVAL, "kerr_params_read: checksum mismatch (corrupted file)");
    return KERR_OK;
}

extern "C" int kerr_surrogate_save(kerr_surrogate *s, const char *path)
{
    if (!s || !path)
        return fail(KERR_EINVAL, "kerr_surrogate_save: NULL argument");
    std::vector<float> p(kL.total);
    int rc = kerr_surrogate_get_params(s, p.data());
    if (rc)
        return rc;
    return kerr_params_write(path, p.data(), (int64_t)p.size());
}

extern "C" int kerr_surrogate_load(const char *path, kerr_surrogate **out)
{
    if (!path || !out)
        return fail(KERR_EINVAL, "kerr_surrogate_load: NULL argument");
    *out = nullptr;
    std::vector<float> p(kL.total);
    int rc = kerr_params_read(path, p.data(), (int64_t)p.size());
    if (rc)
        return rc;
    return kerr_surrogate_create(p.data(), out);
}
