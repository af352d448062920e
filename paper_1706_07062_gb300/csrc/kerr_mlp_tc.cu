// kerr_mlp_tc.cu -- the surrogate's inference forward, all five layers fused
// in one persistent kernel on the 5th-generation tensor cores (tcgen05).
//
// Per 128-row tile (one CTA of 256 threads, one tile at a time):
//   input rows (fp32) -> bf16 tile X [128][16] in shared memory
//   layer 0: D = X W0^T           (1 MMA, M = 128, N = 256, K = 16)
//   layers 1-3: D = A W_l^T       (16 MMAs of K = 16, N = 256)
//   layer 4: D = A W4^T           (16 MMAs, N = 64; 8 outputs used)
// The accumulator D (128 lanes x 256 fp32 columns) lives in tensor memory;
// after each layer the eight warps read it back (tcgen05.ld; warps w and
// w + 4 share TMEM lanes 32 (w % 4) .. + 31 and split the columns), add the
// bias, apply SiLU, round to bf16 and write the next layer's A operand into
// shared memory.  Weights are staged per layer by one bulk TMA copy
// (cp.async.bulk, completion on an mbarrier) from a copy kept in the
// operand layout below, overlapping the previous layer's epilogue.
//
// Operand layout (K-major, no swizzle): a tile of R rows and K columns is
// stored as 8 x 8 "core matrices" of 128 contiguous bytes (8 rows of 16 B);
// byte(r, k) = (r / 8) * (K * 16) + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
// In the MMA's shared-memory descriptor the leading-dimension byte offset is
// the distance between core matrices adjacent in K (128 B) and the
// stride-dimension byte offset the distance between 8-row groups (K * 16 B).
//
// Same arithmetic as the GEMM path (bf16 operands, fp32 accumulation, bias
// and SiLU in fp32, bf16 activations); only the accumulation order differs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kerr_mlp.cuh"
#include "kerr_tc.cuh"

namespace kerr {
namespace mlp {

namespace {

using namespace kerr::tc;

constexpr int TM = 128;   // rows per tile (MMA M)

// Packed weight offset (bf16 elements) of layer l (l = kLayers: the total),
// operand layout.
__host__ __device__ constexpr size_t pack_off(int l)
{
    // layer 0: [256][16]; layers 1-3: [256][256]; layer 4: [64][256]
    return l <= 0 ? 0
                  : (size_t)kHidden * kInPad + (size_t)(l < kLayers ? l - 1 : kLayers - 2) *
                                                   kHidden * kHidden +
                        (l == kLayers ? (size_t)kOutPad * kHidden : 0);
}
static_assert(pack_off(1) == 4096 && pack_off(2) == 4096 + 65536 && pack_off(4) == 4096 + 3 * 65536,
              "packed weight offsets");
static_assert(pack_off(kLayers) == 217088, "packed weight size");

// Shared memory (bytes).
constexpr uint32_t SM_ACT = 0;                               // A operand [128][256]: 64 KB
constexpr uint32_t SM_W = SM_ACT + TM * kHidden * 2;         // W_l [256][256]: 128 KB
constexpr uint32_t SM_X = SM_W + kHidden * kHidden * 2;      // X [128][16]: 4 KB
constexpr uint32_t SM_W0 = SM_X + TM * kInPad * 2;           // W0 [256][16]: 8 KB
constexpr uint32_t SM_BIAS = SM_W0 + kHidden * kInPad * 2;   // 4 x 256 + 64 floats
constexpr uint32_t SM_BAR = SM_BIAS + (4 * kHidden + kOutPad) * 4;
constexpr uint32_t SM_TOTAL = SM_BAR + 64;                   // 2 mbarriers, TMEM slot, flag
static_assert(SM_TOTAL <= 227 * 1024, "shared memory of the fused forward");
static_assert(SM_W % 16 == 0 && SM_X % 16 == 0 && SM_W0 % 16 == 0 && SM_BAR % 8 == 0,
              "bulk-copy and mbarrier alignment");

constexpr uint32_t kTmemCols = 256;          // fp32 accumulator columns (N <= 256)

struct Bias {
    const float *b[kLayers];
};

// Hidden-layer epilogue of one thread: row `row` of the accumulator, columns
// [32 c0, 32 c1) -> bias + SiLU -> bf16 A operand of the next layer.
__device__ __forceinline__ void epilogue_hidden(uint32_t tmem_row, const float *bias,
                                                uint32_t act, int t, int c0, int c1)
{
    const uint32_t row = act + (t >> 3) * (kHidden * 16) + (t & 7) * 16;
#pragma unroll 1
    for (int c = c0; c < c1; ++c) {
        uint32_t v[32];
        tmem_ld32(tmem_row + 32 * c, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = 32 * c + 8 * q + 2 * j;
                const float z0 = __uint_as_float(v[8 * q + 2 * j]) + bias[col];
                const float z1 = __uint_as_float(v[8 * q + 2 * j + 1]) + bias[col + 1];
                w[j] = pack_bf16(silu(z0), silu(z1));
            }
            st_shared_v4(row + (4 * c + q) * 128, w[0], w[1], w[2], w[3]);
        }
    }
}

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads, 1)
    mlp_forward_tc_kernel(const float *__restrict__ in, int64_t n, float *__restrict__ out,
                          const __nv_bfloat16 *__restrict__ wpk, const Bias bias,
                          unsigned *__restrict__ err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int t = threadIdx.x;
    const int warp = t >> 5;
    const int row = t & (TM - 1);      // accumulator row (TMEM lane) of this thread
    const int half = t >> 7;           // column half of the epilogue
    float *sb = reinterpret_cast<float *>(smem + SM_BIAS);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SM_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SM_BAR + 16);
    int *abort_flag = reinterpret_cast<int *>(smem + SM_BAR + 20);
    const uint32_t bar_w = smem_u32(&bars[0]);
    const uint32_t bar_mma = smem_u32(&bars[1]);
    const uint32_t s_act = smem_u32(smem + SM_ACT);
    const uint32_t s_w = smem_u32(smem + SM_W);
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
        mbar_init(bar_w, 1);
        mbar_init(bar_mma, 1);
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
    const uint32_t tmem_row = tmem + ((uint32_t)(32 * (warp & 3)) << 16);

    uint32_t ph_w = 0, ph_mma = 0;
    bool ok = true;
    // W0 stays resident
    if (t == 0) {
        mbar_expect_tx(bar_w, kHidden * kInPad * 2);
        bulk_load(s_w0, wpk + pack_off(0), kHidden * kInPad * 2, bar_w);
    }
    ok = mbar_wait(bar_w, ph_w);
    ph_w ^= 1;

    const int64_t tiles = (n + TM - 1) / TM;
    constexpr uint32_t idesc_h = make_idesc(TM, kHidden);
    constexpr uint32_t idesc_o = make_idesc(TM, kOutPad);
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t r0 = tile * TM;
        if (!ok)
            *abort_flag = 1;
        __syncthreads();
        if (*abort_flag)
            break;
        // W1 into the weight buffer (free: the last tile's MMAs completed)
        if (t == 0 && ok) {
            mbar_expect_tx(bar_w, kHidden * kHidden * 2);
            bulk_load(s_w, wpk + pack_off(1), kHidden * kHidden * 2, bar_w);
        }
        // input tile: row t, columns 0-3 live, 4-15 zero
        if (t < TM) {
            const int64_t r = r0 + t;
            float x[4] = {0.f, 0.f, 0.f, 0.f};
            if (r < n) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    x[j] = in[r * kIn + j];
            }
            const uint32_t xrow = s_x + (t >> 3) * (kInPad * 16) + (t & 7) * 16;
            st_shared_v4(xrow, pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]), 0u, 0u);
            st_shared_v4(xrow + 128, 0u, 0u, 0u, 0u);
        }
        fence_proxy_async();
        fence_before();
        __syncthreads();
        // ---- layer 0 (K = 16): one MMA
        if (t == 0 && ok) {
            fence_after();
            mma_bf16(tmem, make_desc(s_x, 128, kInPad * 16), make_desc(s_w0, 128, kInPad * 16),
                     idesc_h, 0u);
            mma_commit(bar_mma);
        }
        ok = ok && mbar_wait(bar_mma, ph_mma);
        ph_mma ^= 1;
        fence_after();
        epilogue_hidden(tmem_row, sb, s_act, row, 4 * half, 4 * half + 4);
        fence_proxy_async();
        fence_before();
        __syncthreads();
        // ---- hidden layers 1-3 and the output layer
#pragma unroll 1
        for (int l = 1; l < kLayers; ++l) {
            ok = ok && mbar_wait(bar_w, ph_w);      // W_l staged
            ph_w ^= 1;
            const bool last = l == kLayers - 1;
            if (t == 0 && ok) {
                fence_after();
#pragma unroll 1
                for (int s = 0; s < kHidden / 16; ++s)
                    mma_bf16(tmem, make_desc(s_act + s * 256, 128, kHidden * 16),
                             make_desc(s_w + s * 256, 128, kHidden * 16),
                             last ? idesc_o : idesc_h, s > 0 ? 1u : 0u);
                mma_commit(bar_mma);
            }
            ok = ok && mbar_wait(bar_mma, ph_mma);
            ph_mma ^= 1;
            // the weight buffer is free again: stage the next layer's weights
            if (t == 0 && ok && l + 1 < kLayers) {
                const uint32_t bytes = (uint32_t)((pack_off(l + 2) - pack_off(l + 1)) * 2);
                mbar_expect_tx(bar_w, bytes);
                bulk_load(s_w, wpk + pack_off(l + 1), bytes, bar_w);
            }
            fence_after();
            if (!last) {
                epilogue_hidden(tmem_row, sb + l * kHidden, s_act, row, 4 * half,
                                4 * half + 4);
                fence_proxy_async();
            } else if (half == 0) {
                uint32_t v[8];
                tmem_ld8(tmem_row, v);
                const int64_t r = r0 + row;
                if (r < n) {
                    const float *b4 = sb + 4 * kHidden;
                    float4 *o = reinterpret_cast<float4 *>(out + r * kOut);
                    const float4 lo = make_float4(__uint_as_float(v[0]) + b4[0],
                                                  __uint_as_float(v[1]) + b4[1],
                                                  __uint_as_float(v[2]) + b4[2],
                                                  __uint_as_float(v[3]) + b4[3]);
                    const float4 hi = make_float4(__uint_as_float(v[4]) + b4[4],
                                                  __uint_as_float(v[5]) + b4[5],
                                                  __uint_as_float(v[6]) + b4[6],
                                                  __uint_as_float(v[7]) + b4[7]);
                    o[0] = lo;
                    o[1] = hi;
                }
            }
            fence_before();
            __syncthreads();
        }
    }
    if (!ok) {
        // a wait gave up (never expected): flag it, and give whatever this
        // thread may have left in flight one more bounded wait before the
        // tensor memory is freed
        if (err)
            atomicExch(err, 1u);
        if (t == 0) {
            mbar_wait(bar_w, ph_w);
            mbar_wait(bar_mma, ph_mma);
        }
    }
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

// Weights from the bf16 copy ([out][in] per layer) into the operand layout.
struct WOff {
    size_t w[kLayers];
};

__global__ void pack_weights_kernel(const __nv_bfloat16 *__restrict__ wbf, const WOff woff,
                                    __nv_bfloat16 *__restrict__ wpk)
{
    const size_t total = pack_off(kLayers);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < kLayers && i >= pack_off(l + 1))
            ++l;
        const size_t j = i - pack_off(l);
        const int K = in_dim(l);
        const int nrow = (int)(j / K), k = (int)(j % K);
        const size_t dst = pack_off(l) + (size_t)(nrow >> 3) * (K * 8) + (size_t)(k >> 3) * 64 +
                           (nrow & 7) * 8 + (k & 7);
        wpk[dst] = wbf[woff.w[l] + j];
    }
}

} // namespace

size_t packed_weight_elems() { return pack_off(kLayers); }
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
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(
            mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_TOTAL);
        if (e != cudaSuccess)
            return e;
        attr = true;
    }
    Bias b;
    for (int l = 0; l < kLayers; ++l)
        b.b[l] = bias[l];
    const int64_t tiles = (n + TM - 1) / TM;
    const int grid = (int)(tiles < sms ? tiles : sms);
    mlp_forward_tc_kernel<<<grid, kThreads, SM_TOTAL, s>>>(in, n, out, wpk, b, err);
    return cudaGetLastError();
}

} // namespace mlp
} // namespace kerr
