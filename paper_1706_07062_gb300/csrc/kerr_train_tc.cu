// kerr_train_tc.cu -- the surrogate's training step as three tensor-core
// kernels (tcgen05, accumulators in tensor memory).
//
// train_chain_kernel: one CTA per 128-row tile of the batch runs the tile's
// whole chain of nine dependent layers:
//   forward   F0 .. F3: Z_l = A_l W_l^T + b_l, A_{l+1} = bf16(silu(Z_l))
//             F4:       out = A_4 W_4^T + b_4, loss, D_4 = bf16(dL/dout)
//   backward  B4 .. B1: D_{l-1} = bf16((D_l W_l) * silu'(Z_{l-1}))
// Every layer's A operand stays in shared memory, its accumulator in tensor
// memory; the weights stream through four 32 KB slots (K-slices of 64, the
// backward layers' operands transposed at packing time).  The epilogues keep
// what the weight gradients need, in global memory: silu'(Z_l) (fp32), and
// the layer inputs A_l and output gradients D_l transposed.
//
// train_grads_kernel: dW_l = D_l^T A_l and db_l = D_l^T 1 contracted over the
// batch: one CTA per (layer, 128 output features, batch split), the
// transposed operands streamed in 64-row blocks, each split's partial sums
// stored as a full copy of the gradient (no atomics).  The bias gradient is
// one more MMA per K-step against a ones operand, i.e. the column sum of the
// bf16 gradient.
//
// train_adam_kernel: sums the splits' partials in split order (so the
// gradient is deterministic), applies Adam to every parameter and writes the
// row-major bf16 weights and the packed operands of the chain.
//
// Arithmetic as the layer-by-layer GEMM path: bf16 operands, fp32
// accumulation, bias and SiLU in fp32 (hardware exp2 and reciprocal
// approximations), bf16 activations and gradients.
//
// Operand layout (K-major, no swizzle) as in kerr_mlp_tc.cu: a tile of R rows
// and K columns is stored as 8 x 8 core matrices of 128 contiguous bytes,
// byte(r, k) = (r / 8) * (K * 16) + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
// The transposed batch operands of the weight gradients are kept in 64-row
// blocks of that layout, [feature][row]: block b holds rows 64 b .. 64 b + 63
// of every feature, so that any 128 features of one block are one
// contiguous bulk copy.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kerr_mlp.cuh"
#include "kerr_tc.cuh"

namespace kerr {
namespace mlp {

namespace {

using namespace kerr::tc;
using bf16 = __nv_bfloat16;

constexpr int TM = 128;            // rows per tile (MMA M)
constexpr int KS = 64;             // K columns per weight slice
constexpr int kSlices = kHidden / KS;

// ---- packed training weights (bf16 elements)
// forward: W0 [256][16], then layers 1-3 as four [256][64] K-slices and the
// output layer as four [64][64] K-slices (the inference forward's layout);
// backward: W_4^T [256][64], then W_3^T, W_2^T, W_1^T as four [256][64]
// K-slices each (B[n][k] = W_l[k][n]).
constexpr size_t kFwdElems = (size_t)kHidden * kInPad + 3 * kSlices * (size_t)kHidden * KS +
                             kSlices * (size_t)kOutPad * KS;
__host__ __device__ constexpr size_t fwd_off(int l, int s)
{
    return (size_t)kHidden * kInPad +
           (l < kLayers - 1 ? (size_t)(l - 1) * kSlices * kHidden * KS + (size_t)s * kHidden * KS
                            : 3 * (size_t)kSlices * kHidden * KS + (size_t)s * kOutPad * KS);
}
__host__ __device__ constexpr size_t bwd_off(int l, int s)
{
    return kFwdElems + (l == kLayers - 1 ? 0
                                         : (size_t)kHidden * kOutPad +
                                               (size_t)(3 - l) * kSlices * kHidden * KS +
                                               (size_t)s * kHidden * KS);
}
constexpr size_t kPackedElems = bwd_off(1, kSlices);
static_assert(kFwdElems == 217088 && fwd_off(4, 0) == 4096 + 3 * 65536, "forward packing");
static_assert(kPackedElems == kFwdElems + 16384 + 3 * 65536, "backward packing");

// Element (r, k) of an [R][K] operand tile in the core-matrix layout.
__host__ __device__ constexpr size_t cm(int r, int k, int K)
{
    return (size_t)(r >> 3) * (K * 8) + (size_t)(k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// ---- transposed batch operands: features F, 64-row blocks
__host__ __device__ constexpr size_t blk(int f, int64_t r, int F)
{
    return (size_t)(r >> 6) * ((size_t)F * 64) + cm(f, (int)(r & 63), 64);
}
// layer inputs A_l^T (l = 0: the 16 padded input features; 1-4: 256)
__host__ __device__ constexpr size_t ht_base(int l, int64_t cap)
{
    return l == 0 ? 0 : (size_t)cap * kInPad + (size_t)(l - 1) * cap * kHidden;
}
__host__ __device__ constexpr int ht_feat(int l) { return l == 0 ? kInPad : kHidden; }
// output gradients D_l^T (l = 0-3: 256 features; 4: the 64 padded outputs)
__host__ __device__ constexpr size_t dt_base(int l, int64_t cap) { return (size_t)l * cap * kHidden; }
__host__ __device__ constexpr int dt_feat(int l) { return l == kLayers - 1 ? kOutPad : kHidden; }

// Weights from the bf16 copy ([out][in] per layer) into the packed training
// operands: one thread per source element, written to its forward and (for
// layers 1-4) its backward position.
struct WOff {
    size_t w[kLayers];
};

__global__ void train_pack_kernel(const bf16 *__restrict__ wbf, const WOff woff,
                                  bf16 *__restrict__ wtp)
{
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
        const int o = (int)(j / K), k = (int)(j % K);      // W_l[o][k]
        const bf16 v = wbf[woff.w[l] + j];
        if (l == 0) {
            wtp[cm(o, k, kInPad)] = v;
        } else {
            wtp[fwd_off(l, k / KS) + cm(o, k % KS, KS)] = v;
            // backward operand B[n = k][kk = o] in K-slices over o
            wtp[bwd_off(l, o / KS) + cm(k, o % KS, KS)] = v;
        }
    }
}

} // namespace

size_t train_sp_elems(int64_t cap) { return (size_t)4 * cap * kHidden; }
size_t train_ht_elems(int64_t cap) { return ht_base(kLayers, cap); }
size_t train_dt_elems(int64_t cap) { return dt_base(kLayers - 1, cap) + (size_t)cap * kOutPad; }
size_t train_packed_elems() { return kPackedElems; }

cudaError_t train_zero_bufs(TrainBufs b, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(b.ht, 0, train_ht_elems(b.cap) * sizeof(bf16), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b.dt, 0, train_dt_elems(b.cap) * sizeof(bf16), s);
    return e;
}

cudaError_t train_pack(const bf16 *wbf, const size_t woff[kLayers], bf16 *wtp, cudaStream_t s)
{
    WOff o;
    for (int l = 0; l < kLayers; ++l)
        o.w[l] = woff[l];
    train_pack_kernel<<<256, 256, 0, s>>>(wbf, o, wtp);
    return cudaGetLastError();
}

// ===========================================================================
// train_chain_kernel
// ===========================================================================
namespace {

constexpr int kCSlots = 4;                                    // weight-slice buffers
constexpr uint32_t kSlotBytes = kHidden * KS * 2;             // 32 KB
constexpr int kChainLayers = 9;                               // F0-F4, B4-B1
constexpr int kChainSlices = 3 * kSlices + kSlices + 1 + 3 * kSlices;   // per tile

// Shared memory (bytes) of the chain kernel.
constexpr uint32_t C_ACT = 0;                                 // A operand [128][256]: 64 KB
constexpr uint32_t C_SLOT = C_ACT + TM * kHidden * 2;         // 4 x 32 KB
constexpr uint32_t C_W0 = C_SLOT + kCSlots * kSlotBytes;      // W0 [256][16]: 8 KB
constexpr uint32_t C_BIAS = C_W0 + kHidden * kInPad * 2;      // 4 x 256 + 64 floats
constexpr uint32_t C_BAR = C_BIAS + (4 * kHidden + kOutPad) * 4;
// barriers: full[4], empty[4], accfull, actready, w0, final; TMEM slot; abort flag
constexpr int kCBars = 2 * kCSlots + 4;
constexpr uint32_t C_TOTAL = C_BAR + kCBars * 8 + 8 + 8;
static_assert(C_TOTAL <= 227 * 1024, "shared memory of the chain kernel");
static_assert(C_SLOT % 1024 == 0 && C_W0 % 16 == 0 && C_BIAS % 16 == 0 && C_BAR % 8 == 0,
              "bulk-copy, vector-load and mbarrier alignment");
constexpr int kCMmaWarp = 1;              // warp 0: producer lanes 0-3 (one per slot)
constexpr int kCEpiWarp0 = 2;             // warps 2-17: epilogue
constexpr int kCThreads = 32 * kCEpiWarp0 + 512;
constexpr int kCEpi = 512;

struct Biases {
    const float *b[kLayers];
};

// Weight slice i of a tile's schedule: F1-F3 (four [256][64] slices each),
// F4 (four [64][64]), B4 (one [256][64]: K = 64), B3-B1 (four each).
__device__ __forceinline__ void chain_slice(int i, size_t &off, uint32_t &bytes)
{
    if (i < 3 * kSlices) {
        off = fwd_off(1 + i / kSlices, i % kSlices);
        bytes = kSlotBytes;
    } else if (i < 4 * kSlices) {
        off = fwd_off(kLayers - 1, i - 3 * kSlices);
        bytes = kOutPad * KS * 2;
    } else if (i == 4 * kSlices) {
        off = bwd_off(kLayers - 1, 0);
        bytes = kSlotBytes;
    } else {
        const int j = i - 4 * kSlices - 1;
        off = bwd_off(3 - j / kSlices, j % kSlices);
        bytes = kSlotBytes;
    }
}

// Named barrier 1 over the sixteen epilogue warps (the producer and MMA
// warps never take part).
__device__ __forceinline__ void epi_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kCEpi) : "memory");
}

// The same barrier with a vote: true for every epilogue thread iff p holds
// for all of them.  Every wait outcome goes through it, so that the warps
// leave their loops together and never strand one another at a barrier.
__device__ __forceinline__ bool epi_all(bool p)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred q, rp;\n\t"
                 "setp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.and.pred rp, 1, %2, q;\n\t"
                 "selp.u32 %0, 1, 0, rp;\n\t}\n"
                 : "=r"(r)
                 : "r"((uint32_t)p), "n"(kCEpi)
                 : "memory");
    return r != 0;
}

// silu'(Z_l) of (row r, features f .. f + 3) in [l][feature / 4][row][4]
// floats: the 32 rows of a warp read or write 512 contiguous bytes.
__device__ __forceinline__ size_t sp_at(int l, int f, int64_t r, int64_t cap)
{
    return (((size_t)l * (kHidden / 4) + (f >> 2)) * cap + r) * 4;
}

// The tile's A operand ([128][256] bf16 in shared memory) transposed into the
// 64-row blocks of a batch operand (256 features): 512 8 x 8 matrices, four
// per ldmatrix.trans, which leaves each lane two rows of one feature, stored
// as one 4-byte word (a warp's store covers 128 contiguous bytes).  ew: the
// epilogue warp (0-15); dst: the operand's base; tile: the tile index.
__device__ __forceinline__ void export_transposed(uint32_t act, uint32_t *__restrict__ dst,
                                                  int64_t tile, int ew, int lane)
{
#pragma unroll 2
    for (int it = 0; it < 8; ++it) {
        const int mi = (ew * 8 + it) * 4;               // four matrices of one row group
        const int ma = mi + (lane >> 3);                // the matrix this lane addresses
        const uint32_t addr = act + (ma >> 5) * (kHidden * 16) + (ma & 31) * 128 + (lane & 7) * 16;
        uint32_t v[4];
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                     : "r"(addr)
                     : "memory");
        const int rr = 8 * (mi >> 5) + 2 * (lane & 3);  // tile row of the pair's first element
        const int64_t r = tile * TM + rr;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int f = 8 * ((mi + k) & 31) + (lane >> 2);
            dst[blk(f, r, kHidden) >> 1] = v[k];
        }
    }
}

__device__ __forceinline__ uint16_t bf16_bits(float x)
{
    const bf16 h = __float2bfloat16(x);
    return *reinterpret_cast<const uint16_t *>(&h);
}

// Input row `t` (< 128) of tile `tile` as the layer-0 A operand ([128][16],
// columns 4-15 zero) at `act`, and its 4 live features into A_0^T.
__device__ __forceinline__ void chain_stage_x(const float *__restrict__ in, int64_t rows,
                                              int64_t r0, int64_t tile, int t, uint32_t act,
                                              uint16_t *__restrict__ ht0)
{
    const int64_t r = tile * TM + t;
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    if (r < rows) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            x[j] = in[(r0 + r) * kIn + j];
    }
    const uint32_t xrow = act + (t >> 3) * (kInPad * 16) + (t & 7) * 16;
    st_shared_v4(xrow, pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]), 0u, 0u);
    st_shared_v4(xrow + 128, 0u, 0u, 0u, 0u);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        ht0[blk(j, r, kInPad)] = bf16_bits(x[j]);
}

} // namespace

namespace {

__global__ void __launch_bounds__(kCThreads, 1)
    train_chain_kernel(const float *__restrict__ in, const float *__restrict__ tgt,
                       const float *__restrict__ msk, int64_t rows,
                       const StepCtl *__restrict__ ctl, float *__restrict__ loss_sum,
                       const Biases bias, const bf16 *__restrict__ wtp, const TrainBufs bufs,
                       unsigned *__restrict__ err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int t = threadIdx.x;
    const int warp = t >> 5;
    const int lane = t & 31;
    float *sb = reinterpret_cast<float *>(smem + C_BIAS);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + C_BAR + kCBars * 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + C_BAR + kCBars * 8 + 8);
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    const int B_FULL = 0, B_EMPTY = kCSlots, B_ACC = 2 * kCSlots, B_ACT = 2 * kCSlots + 1,
              B_W0 = 2 * kCSlots + 2, B_FIN = 2 * kCSlots + 3;
    const uint32_t s_act = smem_u32(smem + C_ACT);
    const uint32_t s_slot = smem_u32(smem + C_SLOT);
    const uint32_t s_w0 = smem_u32(smem + C_W0);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        for (int i = 0; i < kCSlots; ++i) {
            mbar_init(bar(B_FULL + i), 1);
            mbar_init(bar(B_EMPTY + i), 1);
        }
        mbar_init(bar(B_ACC), 1);
        mbar_init(bar(B_ACT), kCEpi);
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

    const int64_t ntiles = (rows + TM - 1) / TM;
    const int64_t r0 = ctl ? ctl->r0 : 0;
    bool ok = true;

    if (warp == 0) {
        // ---- producer: lane p issues the copies of the slices that go
        // through slot p (bulk copies of one thread complete one after
        // another, those of different threads overlap).  The lanes walk the
        // slices together in the MMA's order: at slice k only lane k % 4 waits
        // (for the slot's previous slice, which the MMAs free in order) and
        // issues, so no lane ever waits on a later slice while an earlier
        // one is still to be issued.  W0 once, from lane 0.
        const int p = lane;
        if (p == 0) {
            mbar_expect_tx(bar(B_W0), kHidden * kInPad * 2);
            bulk_load(s_w0, wtp, kHidden * kInPad * 2, bar(B_W0));
        }
        uint32_t k = 0, issued = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            for (int i = 0; i < kChainSlices && ok; ++i, ++k) {
                const int owner = (int)(k % kCSlots);
                if (p == owner) {
                    const uint32_t use = k / kCSlots;
                    if (use >= 1 && !wait_or_abort(bar(B_EMPTY + p), (use - 1) & 1, abort_flag)) {
                        ok = false;
                    } else {
                        size_t off;
                        uint32_t bytes;
                        chain_slice(i, off, bytes);
                        mbar_expect_tx(bar(B_FULL + p), bytes);
                        bulk_load(s_slot + p * kSlotBytes, wtp + off, bytes, bar(B_FULL + p));
                        issued = use + 1;
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, owner) != 0;
            }
        }
        if (!ok && lane == 0)
            *abort_flag = 1;
        // the copies issued have landed before the CTA can exit (already
        // true unless a wait gave up)
        if (p < kCSlots && issued > 0)
            mbar_wait(bar(B_FULL + p), (issued - 1) & 1);
        if (p == 0)
            mbar_wait(bar(B_W0), 0);
    } else if (warp == kCMmaWarp) {
        // ---- MMA issuer: per tile F0 (one MMA against the resident W0), then
        // F1-F3, F4, B4, B3-B1 on the streamed slices
        if (lane == 0) {
            uint32_t k = 0, ph_act = 0;
            ok = wait_or_abort(bar(B_W0), 0, abort_flag);
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                for (int L = 0; L < kChainLayers && ok; ++L) {
                    if (!wait_or_abort(bar(B_ACT), ph_act, abort_flag)) {
                        ok = false;
                        break;
                    }
                    ph_act ^= 1;
                    fence_after();
                    if (L == 0) {
                        mma_bf16(tmem, make_desc(s_act, 128, kInPad * 16),
                                 make_desc(s_w0, 128, kInPad * 16), make_idesc(TM, kHidden), 0u);
                    } else {
                        const bool b4 = L == 5;                 // A: D_4 [128][64], K = 64
                        const int ns = b4 ? 1 : kSlices;
                        const uint32_t idesc =
                            L == 4 ? make_idesc(TM, kOutPad) : make_idesc(TM, kHidden);
                        const uint32_t asbo = b4 ? KS * 16 : kHidden * 16;
                        for (int s = 0; s < ns; ++s, ++k) {
                            const uint32_t slot = k % kCSlots;
                            if (!wait_or_abort(bar(B_FULL + slot), (k / kCSlots) & 1,
                                               abort_flag)) {
                                ok = false;
                                break;
                            }
                            fence_after();
                            const uint32_t w = s_slot + slot * kSlotBytes;
#pragma unroll
                            for (int j = 0; j < KS / 16; ++j)
                                mma_bf16(tmem, make_desc(s_act + s * (KS / 8) * 128 + j * 256, 128, asbo),
                                         make_desc(w + j * 256, 128, KS * 16), idesc,
                                         (s > 0 || j > 0) ? 1u : 0u);
                            mma_commit(bar(B_EMPTY + slot));
                        }
                    }
                    if (ok)
                        mma_commit(bar(B_ACC));
                }
            }
            if (!ok)
                *abort_flag = 1;
            // every MMA issued has completed before the tensor memory is freed
            mma_commit(bar(B_FIN));
            mbar_wait(bar(B_FIN), 0);
        }
    } else {
        // ---- epilogue: sixteen warps; the four warps of a TMEM lane quarter
        // take 64 of the 256 columns each (two 32-column chunks)
        const int ew = warp - kCEpiWarp0;
        const int et = t - 32 * kCEpiWarp0;             // 0 .. 511
        const int quarter = warp & 3;
        const int colq = ew >> 2;
        const int row = 32 * quarter + lane;            // accumulator row of this thread
        const uint32_t acc_row = tmem + ((uint32_t)(32 * quarter) << 16);
        const uint32_t arow = s_act + (row >> 3) * (kHidden * 16) + (row & 7) * 16;
        const int64_t cap = bufs.cap;
        uint16_t *ht = reinterpret_cast<uint16_t *>(bufs.ht);
        uint16_t *dt = reinterpret_cast<uint16_t *>(bufs.dt);
        const float inv_n = 1.0f / (float)rows;
        float *lsum = loss_sum + (ctl ? ctl->ep : 0);
        uint32_t ph = 0;
        auto wait_acc = [&]() -> bool {
            if (!wait_or_abort(bar(B_ACC), ph, abort_flag))
                return false;
            ph ^= 1;
            fence_after();
            return true;
        };
        auto publish = [&]() {
            fence_proxy_async();
            fence_before();
            mbar_arrive(bar(B_ACT));
        };
        if ((int64_t)blockIdx.x < ntiles) {
            if (et < TM)
                chain_stage_x(in, rows, r0, blockIdx.x, et, s_act, ht + ht_base(0, cap));
            publish();
        }
        // Per layer: wait for the accumulator, write the next A operand into
        // shared memory (and silu'(Z) to global memory), synchronise the
        // epilogue warps, publish the operand to the MMA warp, then export it
        // transposed into global memory and synchronise again before the
        // next layer overwrites it.
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int64_t r = tile * TM + row;          // batch row of this thread
            // F0-F3: bias and SiLU
            for (int l = 0; l < kLayers - 1 && ok; ++l) {
                if (!epi_all(wait_acc())) {
                    ok = false;
                    break;
                }
                const float *bl = sb + l * kHidden;
#pragma unroll 1
                for (int c = 2 * colq; c < 2 * colq + 2; ++c) {
                    uint32_t v[32];
                    tmem_ld32(acc_row + 32 * c, v);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int f0 = 32 * c + 8 * q;
                        const float4 b0 = *reinterpret_cast<const float4 *>(bl + f0);
                        const float4 b1 = *reinterpret_cast<const float4 *>(bl + f0 + 4);
                        const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                        // z = acc + b, sigma = 1 / (1 + 2^(-z log2 e)), h = z sigma,
                        // silu'(z) = sigma (1 + z (1 - sigma)); scalar (the f32x2 pair
                        // form was slower here)
                        float h[8], sp[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float z = __uint_as_float(v[8 * q + j]) + bb[j];
                            const float sg = rcp_approx(1.0f + ex2_approx(-z * kLog2e));
                            h[j] = z * sg;
                            sp[j] = sg * (1.0f + z * (1.0f - sg));
                        }
                        st_shared_v4_relaxed(arow + (4 * c + q) * 128, pack_bf16(h[0], h[1]),
                                             pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]),
                                             pack_bf16(h[6], h[7]));
                        *reinterpret_cast<float4 *>(bufs.sp + sp_at(l, f0, r, cap)) =
                            make_float4(sp[0], sp[1], sp[2], sp[3]);
                        *reinterpret_cast<float4 *>(bufs.sp + sp_at(l, f0 + 4, r, cap)) =
                            make_float4(sp[4], sp[5], sp[6], sp[7]);
                    }
                }
                fence_proxy_async();
                epi_sync();
                publish();
                export_transposed(s_act, reinterpret_cast<uint32_t *>(ht + ht_base(l + 1, cap)),
                                  tile, ew, lane);
                epi_sync();
            }
            if (!ok)
                break;
            // F4: outputs, the row's loss and its gradient D_4 (bf16): the A
            // operand of B4 ([128][64]) and transposed into global memory
            if (!epi_all(wait_acc())) {
                ok = false;
                break;
            }
            if (colq == 0) {
                uint32_t v[8];
                tmem_ld8(acc_row, v);
                float dv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float lrow = 0.0f;
                if (r < rows) {
                    const float *b4 = sb + 4 * kHidden;
                    const float *y = tgt + (r0 + r) * kOut;
                    const float *m = msk + (r0 + r) * kOut;
                    float o[kOut];
#pragma unroll
                    for (int j = 0; j < kOut; ++j)
                        o[j] = __uint_as_float(v[j]) + b4[j];
                    const float z = o[0];
                    const float spl = z > 0.f ? z + log1pf(__expf(-z)) : log1pf(__expf(z));
                    lrow = spl - y[0] * z;
                    const float sig = 1.0f / (1.0f + __expf(-z));
                    dv[0] = (sig - y[0]) * inv_n;
#pragma unroll
                    for (int j = 1; j < kOut; ++j) {
                        const float e = m[j] * (o[j] - y[j]);
                        lrow += e * (o[j] - y[j]);
                        dv[j] = 2.0f * e * inv_n;
                    }
                }
                const uint32_t pp[4] = {pack_bf16(dv[0], dv[1]), pack_bf16(dv[2], dv[3]),
                                        pack_bf16(dv[4], dv[5]), pack_bf16(dv[6], dv[7])};
                const uint32_t drow = s_act + (row >> 3) * (KS * 16) + (row & 7) * 16;
                st_shared_v4_relaxed(drow, pp[0], pp[1], pp[2], pp[3]);
#pragma unroll
                for (int kc = 1; kc < KS / 8; ++kc)
                    st_shared_v4_relaxed(drow + kc * 128, 0u, 0u, 0u, 0u);
                uint16_t *d4 = dt + dt_base(kLayers - 1, cap);
#pragma unroll
                for (int j = 0; j < kOut; ++j)
                    d4[blk(j, r, kOutPad)] = (uint16_t)(pp[j >> 1] >> (16 * (j & 1)));
                // the batch mean: a warp sum, one atomic per warp
#pragma unroll
                for (int o2 = 16; o2 > 0; o2 >>= 1)
                    lrow += __shfl_xor_sync(0xffffffffu, lrow, o2);
                if (lane == 0)
                    atomicAdd(lsum, lrow * inv_n);
            }
            publish();
            // B4 .. B1: D_lz = bf16(acc * silu'(Z_lz)) for lz = 3 .. 0, the A
            // operand of the next backward layer (lz > 0), exported transposed
            for (int lz = kLayers - 2; lz >= 0 && ok; --lz) {
                float4 s4[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)             // in flight during the wait
                    s4[i] = *reinterpret_cast<const float4 *>(
                        bufs.sp + sp_at(lz, 64 * colq + 4 * i, r, cap));
                if (!epi_all(wait_acc())) {
                    ok = false;
                    break;
                }
#pragma unroll 1
                for (int c = 2 * colq; c < 2 * colq + 2; ++c) {
                    if (c != 2 * colq) {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            s4[i] = *reinterpret_cast<const float4 *>(
                                bufs.sp + sp_at(lz, 32 * c + 4 * i, r, cap));
                    }
                    uint32_t v[32];
                    tmem_ld32(acc_row + 32 * c, v);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float sp[8] = {s4[2 * q].x,     s4[2 * q].y,     s4[2 * q].z,
                                             s4[2 * q].w,     s4[2 * q + 1].x, s4[2 * q + 1].y,
                                             s4[2 * q + 1].z, s4[2 * q + 1].w};
                        float d[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            d[j] = __uint_as_float(v[8 * q + j]) * sp[j];
                        st_shared_v4_relaxed(arow + (4 * c + q) * 128, pack_bf16(d[0], d[1]),
                                             pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]),
                                             pack_bf16(d[6], d[7]));
                    }
                }
                fence_proxy_async();
                epi_sync();
                if (lz > 0)
                    publish();
                export_transposed(s_act, reinterpret_cast<uint32_t *>(dt + dt_base(lz, cap)),
                                  tile, ew, lane);
                epi_sync();
            }
            if (!ok)
                break;
            // the next tile's input rows (B1's MMA, the last reader of the A
            // operand, has completed; the last export is done)
            const int64_t nt = tile + gridDim.x;
            if (nt < ntiles) {
                if (et < TM)
                    chain_stage_x(in, rows, r0, nt, et, s_act, ht + ht_base(0, cap));
                publish();
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256)
                     : "memory");
    }
}

} // namespace

// ===========================================================================
// train_grads_kernel
// ===========================================================================
namespace {

constexpr int kGStages = 4;
constexpr uint32_t G_ABYTES = TM * KS * 2;               // 128 features x 64 rows: 16 KB
constexpr uint32_t G_BBYTES = kHidden * KS * 2;          // 256 features x 64 rows: 32 KB
constexpr uint32_t G_STAGE = G_ABYTES + G_BBYTES;
constexpr uint32_t G_ONES = kGStages * G_STAGE;          // ones operand [16][64]: 2 KB
constexpr uint32_t G_BAR = G_ONES + 16 * KS * 2;
// barriers: full[4], empty[4], accfull, final; TMEM slot; abort flag
constexpr int kGBars = 2 * kGStages + 2;
constexpr uint32_t G_TOTAL = G_BAR + kGBars * 8 + 8 + 8;
static_assert(G_TOTAL <= 227 * 1024, "shared memory of the gradient kernel");
constexpr int kGThreads = 64 + 256;       // producer warp, MMA warp, 8 epilogue warps
constexpr int kGTiles = 9;                // (layer, 128 output features) tiles
constexpr int kGMaxSplits = 16;

struct GOff {
    size_t w[kLayers], b[kLayers];
};

// Gradient tile i: layers 1-3 two each (output features 0-127, 128-255),
// layer 0 two (16 input features), the output layer one (64 features).
__device__ __forceinline__ void grad_tile(int i, int &l, int &m0)
{
    if (i < 6) {
        l = 1 + i / 2;
        m0 = TM * (i % 2);
    } else if (i < 8) {
        l = 0;
        m0 = TM * (i - 6);
    } else {
        l = kLayers - 1;
        m0 = 0;
    }
}

__global__ void __launch_bounds__(kGThreads, 1)
    train_grads_kernel(const TrainBufs bufs, int64_t nblk, int splits, float *__restrict__ part,
                       size_t np, const GOff off, unsigned *__restrict__ err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int t = threadIdx.x;
    const int warp = t >> 5;
    const int lane = t & 31;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + G_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + G_BAR + kGBars * 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + G_BAR + kGBars * 8 + 8);
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    const int B_FULL = 0, B_EMPTY = kGStages, B_ACC = 2 * kGStages, B_FIN = 2 * kGStages + 1;
    const uint32_t s_stage = smem_u32(smem);
    const uint32_t s_ones = smem_u32(smem + G_ONES);

    int l, m0;
    grad_tile(blockIdx.x / splits, l, m0);
    const int split = blockIdx.x % splits;
    const int64_t kb0 = nblk * split / splits, kb1 = nblk * (split + 1) / splits;
    const int nk = (int)(kb1 - kb0);
    const int Fo = dt_feat(l), Fi = ht_feat(l);
    const uint32_t abytes = (uint32_t)min(TM, Fo - m0) * KS * 2;
    const uint32_t bbytes = (uint32_t)Fi * KS * 2;
    const bf16 *A = bufs.dt + dt_base(l, bufs.cap) + cm(m0, 0, KS);
    const bf16 *B = bufs.ht + ht_base(l, bufs.cap);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        for (int i = 0; i < kGStages; ++i) {
            mbar_init(bar(B_FULL + i), 1);
            mbar_init(bar(B_EMPTY + i), 1);
        }
        mbar_init(bar(B_ACC), 1);
        mbar_init(bar(B_FIN), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the ones operand, and zero A rows beyond a narrow layer's features (they
    // only feed accumulator rows that are not stored)
    uint32_t *ones = reinterpret_cast<uint32_t *>(smem + G_ONES);
    for (int i = t; i < 16 * KS / 2; i += blockDim.x)
        ones[i] = 0x3F803F80u;                          // two bf16 1.0
    if (abytes < G_ABYTES) {
        for (int s = 0; s < kGStages; ++s) {
            uint32_t *z = reinterpret_cast<uint32_t *>(smem + s * G_STAGE + abytes);
            for (int i = t; i < (int)(G_ABYTES - abytes) / 4; i += blockDim.x)
                z[i] = 0u;
        }
    }
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        // ---- producer: lane 3 s copies stage s's A block, lanes 3 s + 1 and
        // 3 s + 2 the two halves of its B block (separate threads, so that the
        // copies overlap)
        if (lane < 3 * kGStages) {
            const int s = lane / 3, part_i = lane % 3;
            const uint32_t bhalf = bbytes >= 2 * 16384 ? bbytes / 2 : bbytes;
            uint32_t issued = 0;
            for (int i = s; i < nk && ok; i += kGStages) {
                const uint32_t use = (uint32_t)(i / kGStages);
                if (use >= 1 && !wait_or_abort(bar(B_EMPTY + s), (use - 1) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                const int64_t kb = kb0 + i;
                const uint32_t dst = s_stage + s * G_STAGE;
                if (part_i == 0) {
                    mbar_expect_tx(bar(B_FULL + s), abytes + bbytes);
                    bulk_load(dst, A + (size_t)kb * Fo * KS, abytes, bar(B_FULL + s));
                    issued = use + 1;
                } else if (part_i == 1 || bhalf < bbytes) {
                    const uint32_t o = (uint32_t)(part_i - 1) * bhalf;
                    bulk_load(dst + G_ABYTES + o,
                              reinterpret_cast<const uint8_t *>(B + (size_t)kb * Fi * KS) + o,
                              bhalf, bar(B_FULL + s));
                    issued = use + 1;
                }
            }
            if (!ok)
                *abort_flag = 1;
            if (issued > 0)
                mbar_wait(bar(B_FULL + s), (issued - 1) & 1);
        }
    } else if (warp == 1) {
        // ---- MMA issuer: per 64-row block four K-steps of the weight
        // gradient (N = the layer's input width) and of the bias gradient
        // against the ones operand (N = 16, column 0 read back)
        if (lane == 0) {
            const uint32_t idesc = make_idesc(TM, Fi), idesc1 = make_idesc(TM, 16);
            for (int i = 0; i < nk && ok; ++i) {
                const int s = i % kGStages;
                if (!wait_or_abort(bar(B_FULL + s), (i / kGStages) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t sa = s_stage + s * G_STAGE, sbb = sa + G_ABYTES;
#pragma unroll
                for (int j = 0; j < KS / 16; ++j) {
                    const uint32_t acc = (i > 0 || j > 0) ? 1u : 0u;
                    const uint64_t da = make_desc(sa + j * 256, 128, KS * 16);
                    mma_bf16(tmem, da, make_desc(sbb + j * 256, 128, KS * 16), idesc, acc);
                    mma_bf16(tmem + 256, da, make_desc(s_ones + j * 256, 128, KS * 16), idesc1,
                             acc);
                }
                mma_commit(bar(B_EMPTY + s));
            }
            if (ok && nk > 0)
                mma_commit(bar(B_ACC));
            if (!ok)
                *abort_flag = 1;
            mma_commit(bar(B_FIN));
            mbar_wait(bar(B_FIN), 0);
        }
    } else {
        // ---- epilogue: eight warps; warp w reads accumulator rows
        // 32 (w % 4) .. + 31 (one output feature each) in one column half and
        // stores them as this split's partial gradient (the parameter layout,
        // one copy per split).  Each 32 x 32 block goes through a per-warp
        // tile in the idle stage buffers, so that every store instruction
        // writes 32 consecutive floats of one row.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int mrow0 = m0 + 32 * quarter;            // first output feature of the warp
        const uint32_t acc_row = tmem + ((uint32_t)(32 * quarter) << 16);
        float *tile = reinterpret_cast<float *>(smem) + (warp - 2) * (32 * 33);
        if (nk > 0) {
            if (!wait_or_abort(bar(B_ACC), 0, abort_flag)) {
                ok = false;
            } else {
                fence_after();
                float *pg = part + (size_t)split * np;
                const int ncol = Fi == kHidden ? kHidden / 2 : kInPad;   // this warp's columns
                const int c0 = Fi == kHidden ? half * (kHidden / 2) : 0;
                if (Fi == kHidden || half == 0) {
#pragma unroll 1
                    for (int c = c0; c < c0 + ncol; c += 32) {
                        const int w = min(32, ncol);
                        uint32_t v[32];
                        if (w == 32) {
                            tmem_ld32(acc_row + c, v);
                        } else {
                            tmem_ld8(acc_row + c, v);
                            tmem_ld8(acc_row + c + 8, v + 8);
                        }
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < w)
                                tile[lane * 33 + j] = __uint_as_float(v[j]);
                        __syncwarp();
#pragma unroll 4
                        for (int rr = 0; rr < 32; ++rr) {
                            const int m = mrow0 + rr;
                            if (m < Fo && lane < w)
                                pg[off.w[l] + (size_t)m * Fi + c + lane] = tile[rr * 33 + lane];
                        }
                        __syncwarp();
                    }
                }
                if (half == 0) {
                    uint32_t vb[8];
                    tmem_ld8(acc_row + 256, vb);
                    if (mrow0 + lane < Fo)
                        pg[off.b[l] + mrow0 + lane] = __uint_as_float(vb[0]);
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                     : "memory");
    }
}

} // namespace

// ===========================================================================
// train_adam_kernel
// ===========================================================================
namespace {

// Sum of the splits' partial gradients of four consecutive parameters: every
// split's load is issued before the additions (splits <= kGMaxSplits), so a
// thread keeps up to sixteen 16-byte loads in flight.
__device__ __forceinline__ float4 sum_parts(const float *__restrict__ part, int splits,
                                            size_t np, size_t i)
{
    float4 a[kGMaxSplits];
#pragma unroll
    for (int s = 0; s < kGMaxSplits; ++s)
        if (s < splits)
            a[s] = *reinterpret_cast<const float4 *>(part + (size_t)s * np + i);
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int s = 0; s < kGMaxSplits; ++s)
        if (s < splits) {
            g.x += a[s].x;
            g.y += a[s].y;
            g.z += a[s].z;
            g.w += a[s].w;
        }
    return g;
}

// g = the sum of the partial gradients (four parameters per thread).
__global__ void train_reduce_kernel(const float *__restrict__ part, int splits, size_t np,
                                    float *__restrict__ g)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < np / 4;
         c += (size_t)gridDim.x * blockDim.x)
        *reinterpret_cast<float4 *>(g + 4 * c) = sum_parts(part, splits, np, 4 * c);
}

// Adam with the step's learning rate and bias corrections, four consecutive
// parameters per thread (a weight row segment or biases: every layer's
// offsets and widths are multiples of 8): the gradient is the sum of the
// partials, then w, m, v, the bf16 copy [out][in] and the packed forward
// operand (one 16- or 8-byte store each) and the packed backward operand
// (four 2-byte stores) are written.
__global__ void train_adam_kernel(float *__restrict__ w, const float *__restrict__ part,
                                  int splits, float *__restrict__ m, float *__restrict__ v,
                                  bf16 *__restrict__ wbf, bf16 *__restrict__ wtp, const WOff o,
                                  size_t np, const StepCtl *__restrict__ ctl, float b1, float b2,
                                  float eps)
{
    const float lr = ctl->lr, c1 = ctl->c1, c2 = ctl->c2;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < np / 4;
         c += (size_t)gridDim.x * blockDim.x) {
        const size_t i = 4 * c;
        const float4 w4 = *reinterpret_cast<const float4 *>(w + i);
        const float4 m4 = *reinterpret_cast<const float4 *>(m + i);
        const float4 v4 = *reinterpret_cast<const float4 *>(v + i);
        const float4 g4 = sum_parts(part, splits, np, i);
        float gs[4] = {g4.x, g4.y, g4.z, g4.w}, wv[4] = {w4.x, w4.y, w4.z, w4.w},
              mv[4] = {m4.x, m4.y, m4.z, m4.w}, vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            mv[j] = b1 * mv[j] + (1.0f - b1) * gs[j];
            vv[j] = b2 * vv[j] + (1.0f - b2) * gs[j] * gs[j];
            wv[j] = wv[j] - lr * (mv[j] * c1) / (sqrtf(vv[j] * c2) + eps);
        }
        *reinterpret_cast<float4 *>(w + i) = make_float4(wv[0], wv[1], wv[2], wv[3]);
        *reinterpret_cast<float4 *>(m + i) = make_float4(mv[0], mv[1], mv[2], mv[3]);
        *reinterpret_cast<float4 *>(v + i) = make_float4(vv[0], vv[1], vv[2], vv[3]);
        const uint32_t wb[2] = {pack_bf16(wv[0], wv[1]), pack_bf16(wv[2], wv[3])};
        const uint2 wq = make_uint2(wb[0], wb[1]);
        *reinterpret_cast<uint2 *>(wbf + i) = wq;
        int l = 0;
        while (l + 1 < kLayers && i >= o.w[l + 1])
            ++l;
        const size_t j = i - o.w[l];
        const int K = in_dim(l), N = out_dim(l);
        if (j < (size_t)N * K) {                                // weights, not biases
            const int oo = (int)(j / K), k = (int)(j % K);      // k .. k + 3 in row oo
            if (l == 0) {
                *reinterpret_cast<uint2 *>(wtp + cm(oo, k, kInPad)) = wq;
            } else {
                *reinterpret_cast<uint2 *>(wtp + fwd_off(l, k / KS) + cm(oo, k % KS, KS)) = wq;
                uint16_t *bw = reinterpret_cast<uint16_t *>(wtp + bwd_off(l, oo / KS));
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    bw[cm(k + jj, oo % KS, KS)] = (uint16_t)(wb[jj >> 1] >> (16 * (jj & 1)));
            }
        }
    }
}

} // namespace

cudaError_t train_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(train_chain_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C_TOTAL);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(train_grads_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)G_TOTAL);
    return e;
}

cudaError_t train_chain(const float *in, const float *tgt, const float *msk, int64_t rows,
                        const StepCtl *ctl, float *loss_sum, const float *const bias[kLayers],
                        const bf16 *wtp, TrainBufs b, unsigned *err, int sms, cudaStream_t s)
{
    if (rows <= 0)
        return cudaSuccess;
    if (rows > b.cap || (b.cap % TM) != 0)
        return cudaErrorInvalidValue;
    Biases bb;
    for (int l = 0; l < kLayers; ++l)
        bb.b[l] = bias[l];
    const int64_t ntiles = (rows + TM - 1) / TM;
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    train_chain_kernel<<<grid, kCThreads, C_TOTAL, s>>>(in, tgt, msk, rows, ctl, loss_sum, bb, wtp,
                                                        b, err);
    return cudaGetLastError();
}

int train_splits(int64_t rows, int sms)
{
    const int64_t nblk = 2 * ((rows + TM - 1) / TM);       // 64-row blocks of the batch
    int64_t splits = sms / kGTiles;
    if (splits > kGMaxSplits)
        splits = kGMaxSplits;
    if (splits > nblk)
        splits = nblk;
    return (int)(splits < 1 ? 1 : splits);
}

size_t train_part_elems(size_t np) { return (size_t)kGMaxSplits * np; }

cudaError_t train_grads(TrainBufs b, int64_t rows, float *part, size_t np,
                        const size_t woff[kLayers], const size_t boff[kLayers], unsigned *err,
                        int sms, cudaStream_t s)
{
    if (rows <= 0)
        return cudaSuccess;
    if (rows > b.cap || (b.cap % TM) != 0 || (np % 8) != 0)
        return cudaErrorInvalidValue;
    const int64_t nblk = 2 * ((rows + TM - 1) / TM);
    const int splits = train_splits(rows, sms);
    GOff o;
    for (int l = 0; l < kLayers; ++l) {
        o.w[l] = woff[l];
        o.b[l] = boff[l];
    }
    train_grads_kernel<<<kGTiles * splits, kGThreads, G_TOTAL, s>>>(b, nblk, splits, part, np, o,
                                                                    err);
    return cudaGetLastError();
}

cudaError_t train_reduce(const float *part, int splits, size_t np, float *g, cudaStream_t s)
{
    if ((np % 8) != 0 || splits < 1 || splits > kGMaxSplits)
        return cudaErrorInvalidValue;
    const int64_t blocks = ((int64_t)np / 4 + 255) / 256;
    train_reduce_kernel<<<(int)blocks, 256, 0, s>>>(part, splits, np, g);
    return cudaGetLastError();
}

cudaError_t train_adam(float *w, const float *part, int splits, float *m, float *v, bf16 *wbf,
                       bf16 *wtp, const size_t woff[kLayers], size_t np, const StepCtl *ctl,
                       float b1, float b2, float eps, cudaStream_t s)
{
    if ((np % 8) != 0 || splits < 1 || splits > kGMaxSplits)
        return cudaErrorInvalidValue;
    WOff o;
    for (int l = 0; l < kLayers; ++l)
        o.w[l] = woff[l];
    const int64_t blocks = ((int64_t)np / 4 + 255) / 256;
    train_adam_kernel<<<(int)blocks, 256, 0, s>>>(w, part, splits, m, v, wbf, wtp, o, np, ctl, b1,
                                                  b2, eps);
    return cudaGetLastError();
}

} // namespace mlp
} // namespace kerr
