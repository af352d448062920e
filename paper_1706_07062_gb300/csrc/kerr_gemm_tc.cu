// kerr_gemm_tc.cu -- the surrogate's training GEMMs on the 5th-generation
// tensor cores (tcgen05, accumulator in tensor memory).
//
// C[m][n] = sum_k A[m][k] B[n][k] with both operands bf16 and K-contiguous
// (row strides lda, ldb multiples of 8 elements; K a multiple of 8), fp32
// accumulation, and the fused epilogues of kerr_mlp.cuh (bias, SiLU, bf16
// activations, split-K atomics).
//
// One CTA of 256 threads per 128 x BN output tile (BN = 64, 128 or 256):
//   * all threads stage 64-wide K slices of A (128 rows) and B (BN rows)
//     with 16-byte cp.async copies into the no-swizzle K-major operand layout
//     (8 x 8 core matrices of 128 contiguous bytes; byte(r, k) =
//     (r / 8) * 1024 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2), three
//     buffers, the next two slices' copies in flight while the tensor core
//     works on this one;
//   * thread 0 issues the slice's four MMAs (M = 128, N = BN, K = 16) and
//     commits them to the buffer's mbarrier, whose completion frees the
//     buffer for the copies three slices later;
//   * after the last slice each warp reads 32 accumulator lanes (rows) of
//     one column half back with tcgen05.ld, 32 columns at a time, applies the
//     epilogue and writes through a shared-memory tile, one row segment per
//     instruction.
// Rows of A beyond M, rows of B beyond N and K beyond the split's end are
// staged as zeros; only rows < M and columns < N are written.  Every
// mbarrier wait is bounded: on a time-out the CTA sets *err, stops issuing,
// gives its MMAs one more bounded wait and frees its tensor memory.
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

constexpr int TBM = 128, TBK = 64, TTHREADS = 256;

__device__ __forceinline__ void cp16(uint32_t dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

constexpr int NS = 3;   // operand buffers: slices i + 1 and i + 2 load while MMAs run on i

template <int BN> struct TcShape {
    static constexpr uint32_t A_BYTES = TBM * TBK * 2;              // 16 KB
    static constexpr uint32_t B_BYTES = BN * TBK * 2;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr uint32_t BAR = NS * STAGE;                     // buffers, then barriers
    static constexpr uint32_t TOTAL = BAR + 64;
    static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
    // the epilogue's two per-warp tiles (8 warps x 32 x 33 floats each) reuse
    // the operand buffers
    static_assert(2 * 8 * 32 * 33 * 4 <= BAR, "epilogue tiles fit the operand buffers");
};

// Stage the K slice [k0, min(k0 + 64, ke)) of rows [r0, r0 + R) of X (row
// stride ld, `valid_rows` rows exist) into the operand layout at `dst`.
template <int R>
__device__ __forceinline__ void stage_rows(uint32_t dst, const bf16 *__restrict__ X, int ld,
                                           int r0, int valid_rows, int k0, int ke, int t)
{
#pragma unroll
    for (int c = t; c < R * 8; c += TTHREADS) {
        const int r = c % R, kc = c / R;                // a warp: 32 rows of one K chunk
        const int gr = r0 + r, gk = k0 + kc * 8;
        const bool ok = gr < valid_rows && gk < ke;
        const bf16 *src = ok ? X + (size_t)gr * ld + gk : X;
        cp16(dst + (uint32_t)((r >> 3) * 1024 + kc * 128 + (r & 7) * 16), src, ok);
    }
}

template <int BN, int EPI>
__global__ void __launch_bounds__(TTHREADS)
    gemm_tc_kernel(const bf16 *__restrict__ A, int lda, const bf16 *__restrict__ B, int ldb,
                   int M, int N, int K, int kchunk, EpiArgs e, unsigned *__restrict__ err)
{
    using S = TcShape<BN>;
    extern __shared__ __align__(1024) uint8_t smem[];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(K, kb + kchunk);
    const int nk = ke > kb ? (ke - kb + TBK - 1) / TBK : 0;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S::BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + S::BAR + 8 * NS);
    const uint32_t s0 = smem_u32(smem);
    const uint32_t bar0 = smem_u32(&bars[0]);       // barrier of buffer b: bar0 + 8 b

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(S::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        for (int b = 0; b < NS; ++b)
            mbar_init(bar0 + 8 * b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t idesc = make_idesc(TBM, BN);

    // slice i lives in buffer i % NS; its MMAs commit to that buffer's
    // mbarrier, completing phase i / NS there
    auto stage = [&](int i) {
        const uint32_t dst = s0 + (uint32_t)(i % NS) * S::STAGE;
        const int k0 = kb + i * TBK;
        stage_rows<TBM>(dst, A, lda, m0, M, k0, ke, t);
        stage_rows<BN>(dst + S::A_BYTES, B, ldb, n0, N, k0, ke, t);
    };
    auto slice_done = [&](int i) { return mbar_wait(bar0 + 8 * (i % NS), (i / NS) & 1); };
    bool ok = true;
    for (int i = 0; i < NS - 1; ++i) {              // prologue: one commit group per slice
        if (i < nk)
            stage(i);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int i = 0; i < nk; ++i) {
        // refill the buffer of slice i - 1 (its MMAs must have finished) with
        // slice i + NS - 1; empty groups keep the group count per iteration
        const int nxt = i + NS - 1;
        if (nxt < nk) {
            if (i >= 1)
                ok = ok && slice_done(i - 1);
            stage(nxt);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group %0;" ::"n"(NS - 1) : "memory");   // slice i landed
        fence_proxy_async();       // generic-proxy smem writes -> tensor core reads
        fence_before();
        __syncthreads();
        if (t == 0 && ok) {
            fence_after();
            const uint32_t sa = s0 + (uint32_t)(i % NS) * S::STAGE, sb = sa + S::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TBK / 16; ++kk)
                mma_bf16(tmem, make_desc(sa + kk * 256, 128, 1024),
                         make_desc(sb + kk * 256, 128, 1024), idesc,
                         (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(bar0 + 8 * (i % NS));
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (nk > 0)
        ok = ok && slice_done(nk - 1);
    // one decision for the whole CTA: the epilogue's tensor-memory loads are
    // warp-collective
    ok = __syncthreads_and(ok) != 0;
    fence_after();

    // ---- epilogue: warps w and w + 4 read accumulator rows (TMEM lanes)
    // 32 (w % 4) .. + 31 and split the columns in halves.  Each 32-column
    // block goes through a per-warp shared-memory tile (the operand buffers
    // are free now), so that every global store or atomic of the warp covers
    // 32 consecutive columns of one row.
    const int quad = warp & 3, half = warp >> 2;
    const int rw = m0 + 32 * quad;
    const uint32_t trow = tmem + ((uint32_t)(32 * quad) << 16);
    constexpr bool SILU = EPI == EPI_BIAS_SILU || EPI == EPI_BIAS_SILU_BF16;
    float *tile = reinterpret_cast<float *>(smem) + warp * (32 * 33);
    float *tile_a = reinterpret_cast<float *>(smem) + (8 + warp) * (32 * 33);   // SiLU values
    const int myrow = rw + lane;
    if (ok && nk > 0) {
#pragma unroll 1
        for (int cb = half * (BN / 64); cb < (half + 1) * (BN / 64); ++cb) {
            const int c0 = n0 + 32 * cb;
            if (c0 >= N)
                break;                                         // warp-uniform
            // EPI_DSILU: this lane's column of the block's 32 pre-activation
            // rows, all loads in flight before the accumulator is read
            float zr[EPI == EPI_DSILU ? 32 : 1];
            if (EPI == EPI_DSILU) {
                const int zc = min(c0 + lane, N - 1);
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    zr[r] = __ldg(e.Zin + (size_t)min(rw + r, M - 1) * e.ldc + zc);
            }
            uint32_t v[32];
            tmem_ld32(trow + 32 * cb, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float z = __uint_as_float(v[j]);
                if (EPI == EPI_BIAS_F32 || SILU)
                    z += e.bias[min(c0 + j, N - 1)];           // columns >= N are not stored
                tile[lane * 33 + j] = z;
                if (SILU) {
                    const bf16 a = __float2bfloat16(silu(z));
                    tile_a[lane * 33 + j] = __bfloat162float(a);
                    // transposed copy: the warp's 32 rows of one column are
                    // 64 contiguous bytes
                    if (EPI == EPI_BIAS_SILU && e.AoutT && myrow < M && c0 + j < N)
                        e.AoutT[(size_t)(c0 + j) * e.ldT + myrow] = a;
                }
            }
            __syncwarp();
            const int col = c0 + lane;
            if (EPI == EPI_DSILU) {
                // dZ = acc * silu'(Z): row-major (coalesced over columns), the
                // bf16 values back into the tile for the transposed copy, and
                // this warp's column sums for the bias gradient
                float csum = 0.0f;
                if (col < N) {
#pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        const int grow = rw + r;
                        if (grow >= M)
                            break;
                        const float g = tile[r * 33 + lane] * silu_grad(zr[r]);
                        const bf16 gb = __float2bfloat16(g);
                        e.Aout[(size_t)grow * e.lda_out + col] = gb;
                        tile[r * 33 + lane] = __bfloat162float(gb);
                        csum += g;
                    }
                    atomicAdd(e.dbias + col, csum);
                }
                __syncwarp();
                if (myrow < M) {
#pragma unroll 4
                    for (int j = 0; j < 32 && c0 + j < N; ++j)
                        e.AoutT[(size_t)(c0 + j) * e.ldT + myrow] =
                            __float2bfloat16(tile[lane * 33 + j]);
                }
            } else if (col < N) {
#pragma unroll 4
                for (int r = 0; r < 32; ++r) {
                    const int grow = rw + r;
                    if (grow >= M)
                        break;
                    const float z = tile[r * 33 + lane];
                    if (SILU)
                        e.Aout[(size_t)grow * e.lda_out + col] =
                            __float2bfloat16(tile_a[r * 33 + lane]);   // exact: a bf16 value
                    if (EPI != EPI_BIAS_SILU_BF16) {
                        float *cp = e.C + (size_t)grow * e.ldc + col;
                        if (EPI == EPI_F32_ATOMIC)
                            atomicAdd(cp, z);
                        else
                            *cp = z;
                    }
                }
            }
            __syncwarp();
        }
    }
    if (!ok) {
        if (err)
            atomicExch(err, 1u);
        if (t == 0 && nk > 0)
            slice_done(nk - 1);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(S::TMEM_COLS)
                     : "memory");
    }
}

template <int BN, int EPI> cudaError_t set_smem_attr()
{
    return cudaFuncSetAttribute(gemm_tc_kernel<BN, EPI>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<BN>::TOTAL);
}

template <int BN> cudaError_t set_smem_attrs()
{
    cudaError_t e = set_smem_attr<BN, EPI_F32>();
    if (e == cudaSuccess)
        e = set_smem_attr<BN, EPI_BIAS_SILU>();
    if (e == cudaSuccess)
        e = set_smem_attr<BN, EPI_BIAS_F32>();
    if (e == cudaSuccess)
        e = set_smem_attr<BN, EPI_BIAS_SILU_BF16>();
    if (e == cudaSuccess)
        e = set_smem_attr<BN, EPI_F32_ATOMIC>();
    if (e == cudaSuccess)
        e = set_smem_attr<BN, EPI_DSILU>();
    return e;
}

template <int BN, int EPI>
cudaError_t launch(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K,
                   int splits, EpiArgs e, unsigned *err, cudaStream_t s)
{
    using S = TcShape<BN>;
    // whole 64-wide slices per split, every split non-empty
    int kchunk = ((K + splits - 1) / splits + TBK - 1) / TBK * TBK;
    splits = (K + kchunk - 1) / kchunk;
    const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + TBM - 1) / TBM),
                    (unsigned)splits);
    gemm_tc_kernel<BN, EPI><<<grid, TTHREADS, S::TOTAL, s>>>(A, lda, B, ldb, M, N, K, kchunk, e,
                                                             err);
    return cudaGetLastError();
}

template <int EPI>
cudaError_t launch_bn(int bn, const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K,
                      int splits, EpiArgs e, unsigned *err, cudaStream_t s)
{
    if (bn == 64)
        return launch<64, EPI>(A, lda, B, ldb, M, N, K, splits, e, err, s);
    if (bn == 128)
        return launch<128, EPI>(A, lda, B, ldb, M, N, K, splits, e, err, s);
    return launch<256, EPI>(A, lda, B, ldb, M, N, K, splits, e, err, s);
}

} // namespace

cudaError_t gemm_tc_prepare()
{
    cudaError_t e = set_smem_attrs<64>();
    if (e == cudaSuccess)
        e = set_smem_attrs<128>();
    if (e == cudaSuccess)
        e = set_smem_attrs<256>();
    return e;
}

cudaError_t gemm_tc(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K, int epi,
                    EpiArgs e, int splits, unsigned *err, cudaStream_t s)
{
    if (M <= 0 || N <= 0 || K <= 0 || (K & 7) || (lda & 7) || (ldb & 7) || (N & 7) ||
        splits < 1)
        return cudaErrorInvalidValue;
    // N tile: 64 for narrow outputs, else 128 (two tiles across 256 columns
    // give the row-heavy GEMMs twice the CTAs)
    const int bn = N <= 64 ? 64 : 128;
    switch (epi) {
    case EPI_F32:
        return launch_bn<EPI_F32>(bn, A, lda, B, ldb, M, N, K, splits, e, err, s);
    case EPI_BIAS_SILU:
        return launch_bn<EPI_BIAS_SILU>(bn, A, lda, B, ldb, M, N, K, splits, e, err, s);
    case EPI_BIAS_F32:
        return launch_bn<EPI_BIAS_F32>(bn, A, lda, B, ldb, M, N, K, splits, e, err, s);
    case EPI_BIAS_SILU_BF16:
        return launch_bn<EPI_BIAS_SILU_BF16>(bn, A, lda, B, ldb, M, N, K, splits, e, err, s);
    case EPI_F32_ATOMIC:
        return launch_bn<EPI_F32_ATOMIC>(bn, A, lda, B, ldb, M, N, K, splits, e, err, s);
    case EPI_DSILU:
        return launch_bn<EPI_DSILU>(bn, A, lda, B, ldb, M, N, K, splits, e, err, s);
    default:
        return cudaErrorInvalidValue;
    }
}

} // namespace mlp
} // namespace kerr
