// kerr_mlp_tc.cu -- the surrogate's inference forward, all five layers fused
// in one persistent kernel on the 5th-generation tensor cores (tcgen05).
//
// Each CTA works on a pair of 128-row tiles at a time and keeps one fp32
// accumulator per tile in tensor memory (2 x 256 of the 512 columns), so that
// the MMAs of one tile run while the other tile's epilogue reads its
// accumulator back:
//
//   MMA      A0 | B0 | A1 | B1 | A2 | B2 | A3 | B3 | A4 | B4 | (next pair)
//   epilogue      A0 | B0 | A1 | B1 | A2 | B2 | A3 | B3 | A4 | B4
//
// (Xl: layer l of tile X.)  Layer 0 is one MMA (M = 128, N = 256, K = 16)
// against the resident W0; layers 1-4 stream their weights from global
// memory in K-slices of 64 columns ([256][64] bf16 = 32 KB, the output layer
// [64][64]) through two shared-memory slots, each slice consumed by four MMAs
// (K = 16) and released by a tcgen05.commit on the slot's "empty" barrier.
// Warp roles (608 threads):
//   warps 0-1 producers: lane 0 of warp p issues the bulk copies
//             (cp.async.bulk, completion on the slot's "full" mbarrier) of
//             every slice that goes through slot p (on GB300 one issuing
//             warp delivers ~34 B per clock and SM whatever its queue depth,
//             and each further issuing warp adds about as much);
//   warp 2    MMA: one elected lane issues every tcgen05.mma and commit;
//   warps 3-18 epilogue, all sixteen on every accumulator in the MMA's
//             order (the four warps of a TMEM lane quarter take 64 columns
//             each): read the accumulator (tcgen05.ld), add the bias, apply
//             SiLU, round to bf16 and write the next layer's A operand into
//             shared memory (or the 8 outputs to global memory), and signal
//             the MMA warp; during layer 1 they also fetch the input rows of
//             the next pair.  (Two groups of eight warps, one per tile, were
//             slower: the MMA dependencies keep the two tiles' epilogues
//             apart in time, so only half the warps worked at once.)

// Every barrier wait is bounded; a wait that gives up sets the error flag,
// stops its role, and the kernel frees its tensor memory before it exits.
//
// Operand layout (K-major, no swizzle): a tile of R rows and K columns is
// stored as 8 x 8 "core matrices" of 128 contiguous bytes (8 rows of 16 B);
// byte(r, k) = (r / 8) * (K * 16) + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
// In the MMA's shared-memory descriptor the leading-dimension byte offset is
// the distance between core matrices adjacent in K (128 B) and the
// stride-dimension byte offset the distance between 8-row groups (K * 16 B).
//
// Same arithmetic as the GEMM path (bf16 operands, fp32 accumulation, bias
// and SiLU in fp32 with the hardware exp2 and reciprocal approximations, bf16
// activations); only the accumulation order differs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kerr_mlp.cuh"
#include "kerr_tc.cuh"

namespace kerr {
namespace mlp {

namespace {

using namespace kerr::tc;

constexpr int TM = 128;            // rows per tile (MMA M)
constexpr int KS = 64;             // K columns per weight slice
constexpr int kSlices = kHidden / KS;                        // slices per layer (1-4)
constexpr int kSlots = 2;                                    // weight-slice buffers
constexpr uint32_t kSliceBytes = kHidden * KS * 2;           // 32 KB ([256][64] bf16)
constexpr uint32_t kOutSliceBytes = kOutPad * KS * 2;        // 8 KB ([64][64] bf16)

// Packed weights (bf16 elements): W0 [256][16] in the K = 16 layout, then for
// layers 1-4 four K-slices each, every slice [N][64] in the K = 64 layout.
__host__ __device__ constexpr size_t slice_elems(int l) { return (size_t)out_dim(l) * KS; }
__host__ __device__ constexpr size_t slice_off(int l, int s)
{
    return (size_t)kHidden * kInPad +
           (l <= 1 ? 0 : (size_t)(l - 1 < 3 ? l - 1 : 3) * kSlices * slice_elems(1)) +
           (size_t)s * slice_elems(l);
}
constexpr size_t kPackedElems = slice_off(kLayers - 1, kSlices);
static_assert(slice_off(1, 0) == 4096 && slice_off(2, 0) == 4096 + 65536 &&
                  slice_off(4, 0) == 4096 + 3 * 65536,
              "packed weight offsets");
static_assert(kPackedElems == 217088, "packed weight size");

// Shared memory (bytes).
constexpr uint32_t SM_ACT = 0;                                 // 2 x A operand [128][256]: 128 KB
constexpr uint32_t SM_SLOT = SM_ACT + 2 * TM * kHidden * 2;    // 2 x weight slice: 64 KB
constexpr uint32_t SM_X = SM_SLOT + kSlots * kSliceBytes;      // 2 x X [128][16]: 8 KB
constexpr uint32_t SM_W0 = SM_X + 2 * TM * kInPad * 2;         // W0 [256][16]: 8 KB
constexpr uint32_t SM_BIAS = SM_W0 + kHidden * kInPad * 2;     // 4 x 256 + 64 floats
constexpr uint32_t SM_BAR = SM_BIAS + (4 * kHidden + kOutPad) * 4;
// barriers: full[2], empty[2], accfull[2], actready[2], w0, final; TMEM slot; abort flag
constexpr int kBars = 10;
constexpr uint32_t SM_TOTAL = SM_BAR + kBars * 8 + 8 + 8;
static_assert(SM_TOTAL <= 227 * 1024, "shared memory of the fused forward");
static_assert(SM_SLOT % 1024 == 0 && SM_X % 16 == 0 && SM_W0 % 16 == 0 && SM_BAR % 8 == 0,
              "bulk-copy and mbarrier alignment");

constexpr uint32_t kTmemCols = 512;          // two fp32 accumulators of 256 columns
constexpr int kThreads = 32 * (kSlots + 1) + 2 * 256;   // 608
constexpr int kEpiWarp0 = kSlots + 1;          // first epilogue warp
constexpr int kEpiThreads = 512;

struct Bias {
    const float *b[kLayers];
};

// SiLU of two accumulator values with their biases, rounded to a bf16 pair:
// z = acc + b, silu(z) = z / (1 + e^-z) with e^-z = 2^(-z log2 e) and the
// reciprocal from the hardware's approximate exp2 and reciprocal (two MUFU
// operations per element; the MUFU pipe takes 32 per clock and SM).  The
// additions and multiplications run on pairs (one f32x2 instruction for two
// elements).  e^-z beyond the FP32 range gives 1 / inf = 0 and silu = 0 z;
// below 2^-126 it flushes to 0 and silu = z, as the exact values round.
__device__ __forceinline__ uint32_t silu2_bf16(uint32_t a0, uint32_t a1, float b0, float b1)
{
    const float2 z = __fadd2_rn(make_float2(__uint_as_float(a0), __uint_as_float(a1)),
                                make_float2(b0, b1));
    const float2 t = __fmul2_rn(z, make_float2(-kLog2e, -kLog2e));
    const float2 d = __fadd2_rn(make_float2(ex2_approx(t.x), ex2_approx(t.y)),
                                make_float2(1.0f, 1.0f));
    const float2 y = __fmul2_rn(z, make_float2(rcp_approx(d.x), rcp_approx(d.y)));
    return pack_bf16(y.x, y.y);
}

// Hidden-layer epilogue of one thread: accumulator row (TMEM lane) at
// tmem_row, columns [32 c0, 32 c1) -> bias + SiLU -> bf16 A operand row t.
__device__ __forceinline__ void epilogue_hidden(uint32_t tmem_row, const float *bias,
                                                uint32_t act, int t, int c0, int c1)
{
    const uint32_t row = act + (t >> 3) * (kHidden * 16) + (t & 7) * 16;
#pragma unroll 1
    for (int c = c0; c < c1; ++c) {
        float4 b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            b[i] = *reinterpret_cast<const float4 *>(bias + 32 * c + 4 * i);
        uint32_t v[32];
        tmem_ld32(tmem_row + 32 * c, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 lo = b[2 * q], hi = b[2 * q + 1];
            const uint32_t *u = v + 8 * q;
            st_shared_v4_relaxed(row + (4 * c + q) * 128, silu2_bf16(u[0], u[1], lo.x, lo.y),
                      silu2_bf16(u[2], u[3], lo.z, lo.w), silu2_bf16(u[4], u[5], hi.x, hi.y),
                      silu2_bf16(u[6], u[7], hi.z, hi.w));
        }
    }
}

// Input rows of tile `tile` (row t of it, for t < 128) as the bf16 X operand:
// columns 0-3 live, 4-15 zero.  read_x fetches a row from global memory,
// write_x stores it in the operand layout.
__device__ __forceinline__ float4 read_x(const float *__restrict__ in, int64_t n, int64_t tile,
                                         int t)
{
    const int64_t r = tile * TM + t;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < n) {
        x.x = in[r * kIn + 0];
        x.y = in[r * kIn + 1];
        x.z = in[r * kIn + 2];
        x.w = in[r * kIn + 3];
    }
    return x;
}

__device__ __forceinline__ void write_x(float4 x, uint32_t sx, int t)
{
    const uint32_t xrow = sx + (t >> 3) * (kInPad * 16) + (t & 7) * 16;
    st_shared_v4(xrow, pack_bf16(x.x, x.y), pack_bf16(x.z, x.w), 0u, 0u);
    st_shared_v4(xrow + 128, 0u, 0u, 0u, 0u);
}

__global__ void __launch_bounds__(kThreads, 1)
    mlp_forward_tc_kernel(const float *__restrict__ in, int64_t n, float *__restrict__ out,
                          const __nv_bfloat16 *__restrict__ wpk, const Bias bias,
                          unsigned *__restrict__ err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int t = threadIdx.x;
    const int warp = t >> 5;
    const int lane = t & 31;
    float *sb = reinterpret_cast<float *>(smem + SM_BIAS);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SM_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SM_BAR + kBars * 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + SM_BAR + kBars * 8 + 8);
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    const int B_FULL = 0, B_EMPTY = 2, B_ACC = 4, B_ACT = 6, B_W0 = 8, B_FIN = 9;
    const uint32_t s_act = smem_u32(smem + SM_ACT);
    const uint32_t s_slot = smem_u32(smem + SM_SLOT);
    const uint32_t s_x = smem_u32(smem + SM_X);
    const uint32_t s_w0 = smem_u32(smem + SM_W0);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        for (int i = 0; i < kSlots; ++i) {
            mbar_init(bar(B_FULL + i), 1);
            mbar_init(bar(B_EMPTY + i), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar(B_ACC + i), 1);
            mbar_init(bar(B_ACT + i), kEpiThreads);
        }
        mbar_init(bar(B_W0), 1);
        mbar_init(bar(B_FIN), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = t; i < 4 * kHidden + kOutPad; i += blockDim.x)
        sb[i] = i < 4 * kHidden ? bias.b[i / kHidden][i % kHidden]
                                : bias.b[kLayers - 1][i - 4 * kHidden];
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    const int64_t ntiles = (n + TM - 1) / TM;
    const int64_t npairs = (ntiles + 1) / 2;
    bool ok = true;

    if (warp < kSlots) {
        // ---- producers: warp p streams the slices that go through slot p, in
        // the MMA's order (W0 once, from warp 0)
        if (lane == 0) {
            const int p = warp;
            if (p == 0) {
                mbar_expect_tx(bar(B_W0), kHidden * kInPad * 2);
                bulk_load(s_w0, wpk, kHidden * kInPad * 2, bar(B_W0));
            }
            uint32_t k = 0, issued = 0;              // k: slice counter of the MMA's order
            for (int64_t q = blockIdx.x; q < npairs && ok; q += gridDim.x) {
                const int ntile = (2 * q + 1 < ntiles) ? 2 : 1;
                for (int l = 1; l < kLayers && ok; ++l) {
                    const uint32_t bytes = l == kLayers - 1 ? kOutSliceBytes : kSliceBytes;
                    for (int tt = 0; tt < ntile && ok; ++tt) {
                        for (int s = 0; s < kSlices; ++s, ++k) {
                            if (k % kSlots != (uint32_t)p)
                                continue;
                            const uint32_t use = k / kSlots;     // uses of this slot so far
                            if (use >= 1 &&
                                !wait_or_abort(bar(B_EMPTY + p), (use - 1) & 1, abort_flag)) {
                                ok = false;
                                break;
                            }
                            mbar_expect_tx(bar(B_FULL + p), bytes);
                            bulk_load(s_slot + p * kSliceBytes, wpk + slice_off(l, s), bytes,
                                      bar(B_FULL + p));
                            issued = use + 1;
                        }
                    }
                }
            }
            if (!ok)
                *abort_flag = 1;
            // the last copy issued through this slot has landed before the CTA
            // can exit (already true unless a wait gave up)
            if (issued > 0)
                mbar_wait(bar(B_FULL + p), (issued - 1) & 1);
            if (p == 0)
                mbar_wait(bar(B_W0), 0);
        }
    } else if (warp == kSlots) {
        // ---- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc_h = make_idesc(TM, kHidden);
            constexpr uint32_t idesc_o = make_idesc(TM, kOutPad);
            uint32_t k = 0, ph_act[2] = {0, 0};
            ok = wait_or_abort(bar(B_W0), 0, abort_flag);
            for (int64_t q = blockIdx.x; q < npairs && ok; q += gridDim.x) {
                const int ntile = (2 * q + 1 < ntiles) ? 2 : 1;
                for (int l = 0; l < kLayers && ok; ++l) {
                    for (int tt = 0; tt < ntile && ok; ++tt) {
                        if (!wait_or_abort(bar(B_ACT + tt), ph_act[tt], abort_flag)) {
                            ok = false;
                            break;
                        }
                        ph_act[tt] ^= 1;
                        fence_after();
                        const uint32_t acc = tmem + 256u * tt;
                        const uint32_t act = s_act + tt * (TM * kHidden * 2);
                        if (l == 0) {
                            mma_bf16(acc, make_desc(s_x + tt * (TM * kInPad * 2), 128,
                                                    kInPad * 16),
                                     make_desc(s_w0, 128, kInPad * 16), idesc_h, 0u);
                        } else {
                            for (int s = 0; s < kSlices; ++s, ++k) {
                                const uint32_t slot = k % kSlots;
                                if (!wait_or_abort(bar(B_FULL + slot), (k / kSlots) & 1,
                                                   abort_flag)) {
                                    ok = false;
                                    break;
                                }
                                fence_after();
                                const uint32_t w = s_slot + slot * kSliceBytes;
#pragma unroll
                                for (int j = 0; j < KS / 16; ++j)
                                    mma_bf16(acc,
                                             make_desc(act + s * (KS / 8) * 128 + j * 256, 128,
                                                       kHidden * 16),
                                             make_desc(w + j * 256, 128, KS * 16),
                                             l == kLayers - 1 ? idesc_o : idesc_h,
                                             (s > 0 || j > 0) ? 1u : 0u);
                                mma_commit(bar(B_EMPTY + slot));   // slot free once these finish
                            }
                        }
                        if (ok)
                            mma_commit(bar(B_ACC + tt));           // accumulator ready
                    }
                }
            }
            if (!ok)
                *abort_flag = 1;
            // every MMA issued has completed before the tensor memory is freed
            mma_commit(bar(B_FIN));
            mbar_wait(bar(B_FIN), 0);
        }
    } else {
        // ---- epilogue: all sixteen warps serve every accumulator, the two
        // tiles of a pair in the MMA's order (four warps per TMEM lane
        // quarter, each taking 64 of the 256 columns)
        const int ew = warp - kEpiWarp0;                // 0 .. 15
        const int et = t - 32 * kEpiWarp0;              // 0 .. 511
        const int quarter = warp & 3;                   // TMEM lanes 32 quarter ..
        const int colq = ew >> 2;                       // column quarter
        const int row = 32 * quarter + lane;            // accumulator row of this thread
        // input rows: thread et < 256 fetches row et % 128 of tile et / 128
        const int xt = et >> 7;
        const int xr = et & (TM - 1);
        uint32_t ph0 = 0, ph1 = 0;
        // input rows of the first pair
        if (blockIdx.x < npairs) {
            const int ntile = (2 * (int64_t)blockIdx.x + 1 < ntiles) ? 2 : 1;
            if (et < 2 * TM && xt < ntile)
                write_x(read_x(in, n, 2 * (int64_t)blockIdx.x + xt, xr),
                        s_x + xt * (TM * kInPad * 2), xr);
            fence_proxy_async();
            for (int tt = 0; tt < ntile; ++tt)
                mbar_arrive(bar(B_ACT + tt));
        }
        for (int64_t q = blockIdx.x; q < npairs && ok; q += gridDim.x) {
            const int ntile = (2 * q + 1 < ntiles) ? 2 : 1;
            const int64_t qn = q + gridDim.x;           // the next pair of this CTA
            const bool xnext = et < 2 * TM && qn < npairs && 2 * qn + xt < ntiles;
            float4 xn = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int l = 0; l < kLayers && ok; ++l) {
                // the next pair's input rows: read while layer 1's accumulators
                // are computed, stored once the tile's layer-1 accumulator is
                // ready (layer 0's MMA, the reader of X, has then completed)
                if (l == 1 && xnext)
                    xn = read_x(in, n, 2 * qn + xt, xr);
                for (int tt = 0; tt < ntile; ++tt) {
                    if (!wait_or_abort(bar(B_ACC + tt), tt ? ph1 : ph0, abort_flag)) {
                        ok = false;
                        break;
                    }
                    if (tt)
                        ph1 ^= 1;
                    else
                        ph0 ^= 1;
                    fence_after();
                    const uint32_t acc_row =
                        tmem + 256u * tt + ((uint32_t)(32 * quarter) << 16);
                    if (l < kLayers - 1) {
                        epilogue_hidden(acc_row, sb + l * kHidden,
                                        s_act + tt * (TM * kHidden * 2), row, 2 * colq,
                                        2 * colq + 2);
                        if (l == 1 && xnext && xt == tt)
                            write_x(xn, s_x + tt * (TM * kInPad * 2), xr);
                    } else if (colq == 0) {
                        uint32_t v[8];
                        tmem_ld8(acc_row, v);
                        const int64_t r = (2 * q + tt) * TM + row;
                        if (r < n) {
                            const float *b4 = sb + 4 * kHidden;
                            float4 *o = reinterpret_cast<float4 *>(out + r * kOut);
                            o[0] = make_float4(__uint_as_float(v[0]) + b4[0],
                                               __uint_as_float(v[1]) + b4[1],
                                               __uint_as_float(v[2]) + b4[2],
                                               __uint_as_float(v[3]) + b4[3]);
                            o[1] = make_float4(__uint_as_float(v[4]) + b4[4],
                                               __uint_as_float(v[5]) + b4[5],
                                               __uint_as_float(v[6]) + b4[6],
                                               __uint_as_float(v[7]) + b4[7]);
                        }
                    }
                    fence_proxy_async();
                    fence_before();
                    mbar_arrive(bar(B_ACT + tt));
                }
            }
        }
        if (!ok)
            *abort_flag = 1;
    }

    if (!ok && err)
        atomicExch(err, 1u);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

// Weights from the bf16 copy ([out][in] per layer) into the packed operand
// layout: one thread per source element.
struct WOff {
    size_t w[kLayers];
};

__global__ void pack_weights_kernel(const __nv_bfloat16 *__restrict__ wbf, const WOff woff,
                                    __nv_bfloat16 *__restrict__ wpk)
{
    // source elements, layer by layer: [out_dim(l)][in_dim(l)]
    size_t total = 0;
    for (int l = 0; l < kLayers; ++l)
        total += (size_t)out_dim(l) * in_dim(l);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int l = 0;
        size_t j = i;
        while (l + 1 < kLayers && j >= (size_t)out_dim(l) * in_dim(l)) {
            j -= (size_t)out_dim(l) * in_dim(l);
            ++l;
        }
        const int K = in_dim(l);
        const int nrow = (int)(j / K), k = (int)(j % K);
        size_t dst;
        if (l == 0) {
            dst = (size_t)(nrow >> 3) * (kInPad * 8) + (size_t)(k >> 3) * 64 + (nrow & 7) * 8 +
                  (k & 7);
        } else {
            const int s = k / KS, kk = k % KS;
            dst = slice_off(l, s) + (size_t)(nrow >> 3) * (KS * 8) + (size_t)(kk >> 3) * 64 +
                  (nrow & 7) * 8 + (kk & 7);
        }
        wpk[dst] = wbf[woff.w[l] + j];
    }
}

} // namespace

size_t packed_weight_elems() { return kPackedElems; }
int forward_tc_shared_bytes() { return (int)SM_TOTAL; }

cudaError_t pack_weights(const __nv_bfloat16 *wbf, const size_t woff[kLayers],
                         __nv_bfloat16 *wpk, cudaStream_t s)
{
    WOff o;
    for (int l = 0; l < kLayers; ++l)
        o.w[l] = woff[l];
    pack_weights_kernel<<<256, 256, 0, s>>>(wbf, o, wpk);
    return cudaGetLastError();
}

cudaError_t forward_tc(const float *in, int64_t n, float *out, const __nv_bfloat16 *wpk,
                       const float *const bias[kLayers], unsigned *err, int sms, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    // the shared-memory opt-in is per device: set it whenever the device is new
    static int attr_dev = -1;
    if (attr_dev != dev) {
        e = cudaFuncSetAttribute(mlp_forward_tc_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_TOTAL);
        if (e != cudaSuccess)
            return e;
        attr_dev = dev;
    }
    Bias b;
    for (int l = 0; l < kLayers; ++l)
        b.b[l] = bias[l];
    const int64_t tiles = (n + TM - 1) / TM;
    const int64_t pairs = (tiles + 1) / 2;
    const int grid = (int)(pairs < sms ? pairs : sms);
    mlp_forward_tc_kernel<<<grid, kThreads, SM_TOTAL, s>>>(in, n, out, wpk, b, err);
    return cudaGetLastError();
}

} // namespace mlp
} // namespace kerr
