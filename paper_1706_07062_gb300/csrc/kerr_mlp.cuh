// kerr_mlp.cuh -- the surrogate network's kernels: BF16-input / FP32-accumulate
// tensor-core GEMMs with fused epilogues, the loss, and the Adam update.
//
// Network: 4 inputs -> 4 hidden layers of 256 (SiLU) -> 8 outputs.
// Every layer is Y = X W^T + b with X [rows][K] and W [N][K] (K contiguous),
// computed by warp-level tensor-core MMAs (m16n8k16, BF16 operands, FP32
// accumulators).  Input and output widths are padded to the MMA tile:
// K_in = 16 (4 used), N_out = 64 (8 used), padding weights are zero.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kerr {
namespace mlp {

constexpr int kIn = 4, kInPad = 16, kHidden = 256, kLayers = 5, kOut = 8, kOutPad = 64;

// Layer l maps width in_dim(l) to out_dim(l) (padded widths).
__host__ __device__ constexpr int in_dim(int l) { return l == 0 ? kInPad : kHidden; }
__host__ __device__ constexpr int out_dim(int l) { return l == kLayers - 1 ? kOutPad : kHidden; }

// Epilogues of the GEMM.
enum Epi : int {
    EPI_F32 = 0,         // C (fp32) = acc
    EPI_F32_ACC = 1,     // C (fp32) += acc
    EPI_BIAS_SILU = 2,   // Z (fp32) = acc + b;  Aout (bf16) = silu(Z)
    EPI_BIAS_F32 = 3,    // C (fp32) = acc + b
    EPI_BIAS_SILU_BF16 = 4,  // Aout (bf16) = silu(acc + b)  (inference: no Z kept)
    EPI_F32_ATOMIC = 5,  // C (fp32) += acc with atomics (split-K partial sums)
};

struct EpiArgs {
    float *C;            // fp32 output [M][ldc]
    int ldc;
    const float *bias;   // [N]
    __nv_bfloat16 *Aout; // bf16 output [M][lda_out]
    int lda_out;
};

// SiLU with the hardware exp2 and reciprocal approximations (relative error
// ~1e-7, far below the bfloat16 rounding applied to the result).
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ uint32_t ld_b32(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

__device__ __forceinline__ void mma_bf16_16x8x16(float d[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[m][n] = sum_k A(m, k) B(n, k).
//   A(m, k) = A[m * lda + k]   (TA = false)   or A[k * lda + m] (TA = true)
//   B(n, k) = B[n * ldb + k]   (TB = false)   or B[k * ldb + n] (TB = true)
// Tiles: 64 x 64 per block of 128 threads (2 x 2 warps of 32 x 32), K step 32.
// Out-of-range rows/columns/k are read as zero and not written.  Split-K:
// block z covers k in [z kchunk, (z + 1) kchunk) (kchunk a multiple of 32).
// With both operands K-contiguous (K, lda, ldb multiples of 8) the tiles are
// staged by 16-byte cp.async copies into a double buffer, so that the next
// k-step's loads overlap this one's MMAs; transposed operands are staged
// element by element.
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) gemm_bf16(const __nv_bfloat16 *__restrict__ A, int lda,
                                                 const __nv_bfloat16 *__restrict__ B, int ldb,
                                                 int M, int N, int K, int kchunk, EpiArgs e)
{
    constexpr bool ASYNC = !TA && !TB;
    constexpr int NBUF = ASYNC ? 2 : 1;
    __shared__ __align__(16) __nv_bfloat16 As[NBUF][GBM][GBK + GPAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[NBUF][GBN][GBK + GPAD];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r)
                acc[i][j][r] = 0.0f;

    const int kb = blockIdx.z * kchunk;
    const int ke = min(K, kb + kchunk);

    // 16-byte asynchronous staging of one k-tile into buffer `buf`
    auto stage_async = [&](int k0, int buf) {
        for (int c = tid; c < GBM * GBK / 8; c += 128) {
            const int m = c / (GBK / 8), kc = (c % (GBK / 8)) * 8;
            const int gm = m0 + m, gk = k0 + kc;
            const bool ok = gm < M && gk < ke;
            cp_async16(&As[buf][m][kc], ok ? A + (size_t)gm * lda + gk : A, ok);
        }
        for (int c = tid; c < GBN * GBK / 8; c += 128) {
            const int n = c / (GBK / 8), kc = (c % (GBK / 8)) * 8;
            const int gn = n0 + n, gk = k0 + kc;
            const bool ok = gn < N && gk < ke;
            cp_async16(&Bs[buf][n][kc], ok ? B + (size_t)gn * ldb + gk : B, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    auto compute = [&](int buf) {
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm + mt * 16 + g;
                a[mt][0] = ld_b32(&As[buf][r][kk + 2 * t]);
                a[mt][1] = ld_b32(&As[buf][r + 8][kk + 2 * t]);
                a[mt][2] = ld_b32(&As[buf][r][kk + 2 * t + 8]);
                a[mt][3] = ld_b32(&As[buf][r + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int cidx = wn + nt * 8 + g;
                b[nt][0] = ld_b32(&Bs[buf][cidx][kk + 2 * t]);
                b[nt][1] = ld_b32(&Bs[buf][cidx][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
                    mma_bf16_16x8x16(acc[mt][nt], a[mt], b[nt]);
        }
    };

    if constexpr (ASYNC) {
        if (kb < ke)
            stage_async(kb, 0);
        int buf = 0;
        for (int k0 = kb; k0 < ke; k0 += GBK, buf ^= 1) {
            if (k0 + GBK < ke) {
                stage_async(k0 + GBK, buf ^ 1);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncthreads();
            compute(buf);
            __syncthreads();
        }
    } else {
        for (int k0 = kb; k0 < ke; k0 += GBK) {
            for (int i = tid; i < GBM * GBK; i += 128) {
                const int k = TA ? i / GBM : i % GBK, m = TA ? i % GBM : i / GBK;
                const int gm = m0 + m, gk = k0 + k;
                As[0][m][k] = (gm < M && gk < ke)
                                  ? (TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk])
                                  : zero;
            }
            for (int i = tid; i < GBN * GBK; i += 128) {
                const int k = TB ? i / GBN : i % GBK, n = TB ? i % GBN : i / GBK;
                const int gn = n0 + n, gk = k0 + k;
                Bs[0][n][k] = (gn < N && gk < ke)
                                  ? (TB ? B[(size_t)gk * ldb + gn] : B[(size_t)gn * ldb + gk])
                                  : zero;
            }
            __syncthreads();
            compute(0);
            __syncthreads();
        }
    }

    // ---- epilogue: accumulator (row g / g+8, columns 2t, 2t+1) of each tile
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int row = m0 + wm + mt * 16 + g + half * 8;
                if (row >= M)
                    continue;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int col = n0 + wn + nt * 8 + 2 * t + q;
                    if (col >= N)
                        continue;
                    float v = acc[mt][nt][half * 2 + q];
                    if (EPI == EPI_F32) {
                        e.C[(size_t)row * e.ldc + col] = v;
                    } else if (EPI == EPI_F32_ACC) {
                        e.C[(size_t)row * e.ldc + col] += v;
                    } else if (EPI == EPI_F32_ATOMIC) {
                        atomicAdd(&e.C[(size_t)row * e.ldc + col], v);
                    } else if (EPI == EPI_BIAS_F32) {
                        e.C[(size_t)row * e.ldc + col] = v + e.bias[col];
                    } else if (EPI == EPI_BIAS_SILU) {
                        const float z = v + e.bias[col];
                        e.C[(size_t)row * e.ldc + col] = z;
                        e.Aout[(size_t)row * e.lda_out + col] = __float2bfloat16(silu(z));
                    } else {   // EPI_BIAS_SILU_BF16
                        const float z = v + e.bias[col];
                        e.Aout[(size_t)row * e.lda_out + col] = __float2bfloat16(silu(z));
                    }
                }
            }
}

// Fused tensor-core inference forward (kerr_mlp_tc.cu).  Weights are first
// packed from the bf16 copy ([out][in] per layer at offsets woff) into the
// MMA operand layout (packed_weight_elems() bf16); forward_tc then maps
// in [n][4] to out [n][8] on a persistent grid of at most `sms` CTAs.  *err
// becomes nonzero if a pipeline wait gave up (never expected).
size_t packed_weight_elems();
int forward_tc_shared_bytes();
cudaError_t pack_weights(const __nv_bfloat16 *wbf, const size_t woff[kLayers],
                         __nv_bfloat16 *wpk, cudaStream_t s);
cudaError_t forward_tc(const float *in, int64_t n, float *out, const __nv_bfloat16 *wpk,
                       const float *const bias[kLayers], unsigned *err, int sms,
                       cudaStream_t s);

} // namespace mlp
} // namespace kerr
