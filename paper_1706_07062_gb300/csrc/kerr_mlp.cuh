// kerr_mlp.cuh -- the surrogate network's shapes, GEMM epilogues and
// activation, and the entry points of its tensor-core kernels.
//
// Network: 4 inputs -> 4 hidden layers of 256 (SiLU) -> 8 outputs.
// Every layer is Y = X W^T + b with X [rows][K] and W [N][K] (K contiguous),
// bf16 operands and fp32 accumulation on the 5th-generation tensor cores
// (tcgen05): the training GEMMs in kerr_gemm_tc.cu, the fused inference
// forward in kerr_mlp_tc.cu.  Input and output widths are padded to MMA
// shapes: K_in = 16 (4 used), N_out = 64 (8 used), padding weights are zero.
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
    EPI_BIAS_SILU = 2,   // Z (fp32) = acc + b;  Aout (bf16) = silu(Z)
    EPI_BIAS_F32 = 3,    // C (fp32) = acc + b
    EPI_BIAS_SILU_BF16 = 4,  // Aout (bf16) = silu(acc + b)  (inference: no Z kept)
    EPI_F32_ATOMIC = 5,  // C (fp32) += acc with atomics (split-K partial sums)
    EPI_DSILU = 6,       // backward through SiLU: dZ = acc * silu'(Zin) -> Aout (bf16)
                         // and AoutT (transposed), column sums of dZ added to dbias
};

struct EpiArgs {
    float *C;            // fp32 output [M][ldc]
    int ldc;
    const float *bias;   // [N]
    __nv_bfloat16 *Aout; // bf16 output [M][lda_out]
    int lda_out;
    __nv_bfloat16 *AoutT;   // EPI_BIAS_SILU (if set) and EPI_DSILU: the bf16
    int64_t ldT;            // output transposed too, [N][ldT]
    const float *Zin;       // EPI_DSILU: pre-activations [M][ldc]
    float *dbias;           // EPI_DSILU: [N] bias gradient (accumulated)
};

// SiLU with the hardware exp2 and reciprocal approximations (relative error
// ~1e-7, far below the bfloat16 rounding applied to the result).
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// C = A B^T with the epilogue `epi` (an Epi value) on the 5th-generation
// tensor cores (kerr_gemm_tc.cu): A [M][K] and B [N][K] bf16, K-contiguous,
// K, N, lda and ldb multiples of 8; split-K over `splits` CTAs along K (only
// with EPI_F32_ATOMIC).  *err becomes nonzero if a pipeline wait gave up.
cudaError_t gemm_tc(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N,
                    int K, int epi, EpiArgs e, int splits, unsigned *err, cudaStream_t s);
// Sets the GEMM kernels' shared-memory limits (once per device, before any
// gemm_tc call, outside stream capture).
cudaError_t gemm_tc_prepare();

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

// Per-step values of a training run, computed on the device at the start of
// each step (so that every step is the same captured graph): the batch's
// first row, its epoch, the scheduled learning rate and Adam's bias
// corrections.
struct StepCtl {
    long long k;       // steps taken in this run
    long long r0;      // first row of this step's batch
    int ep;            // epoch of this step
    float lr, c1, c2;
};

// Fused training step on the tensor cores (kerr_train_tc.cu): three kernels
// per step.  train_chain runs, for every 128-row tile of the batch in one
// CTA, the five forward layers, the loss and its output gradient, and the
// four backward layers through the hidden weights; train_grads contracts the
// stored activations and gradients over the batch into partial weight and
// bias gradients; train_adam sums them, updates the parameters and refreshes
// the bf16 weights of the forward and training kernels.  Batch-sized buffers of up to `cap` rows (a multiple
// of 128): silu'(Z_l) for l = 0..3 ([4][cap][256] fp32), the layer inputs
// and the output gradients transposed, in 64-row blocks of the tensor-core
// operand layout (bf16).  The parts never written (input features 4-15,
// output-gradient rows 8-63) must be zero: allocate with train_zero_bufs.
struct TrainBufs {
    int64_t cap;
    float *sp;
    __nv_bfloat16 *ht;
    __nv_bfloat16 *dt;
};
size_t train_sp_elems(int64_t cap);
size_t train_ht_elems(int64_t cap);
size_t train_dt_elems(int64_t cap);
cudaError_t train_zero_bufs(TrainBufs b, cudaStream_t s);
// Packed weights of the training kernels: the forward operands (as the
// inference forward's) followed by the transposed operands of the backward
// layers.
size_t train_packed_elems();
cudaError_t train_pack(const __nv_bfloat16 *wbf, const size_t woff[kLayers],
                       __nv_bfloat16 *wtp, cudaStream_t s);
// Shared-memory limits of the training kernels (once per device, outside
// stream capture).
cudaError_t train_prepare();
// rows: batch size (1 .. cap); ctl (may be null): the batch starts at row
// ctl->r0 of in / tgt / msk and the loss mean adds to loss_sum[ctl->ep]
// (else row 0 and loss_sum[0]).  *err becomes nonzero if a pipeline wait
// gave up.
cudaError_t train_chain(const float *in, const float *tgt, const float *msk, int64_t rows,
                        const StepCtl *ctl, float *loss_sum, const float *const bias[kLayers],
                        const __nv_bfloat16 *wtp, TrainBufs b, unsigned *err, int sms,
                        cudaStream_t s);
// The batch's weight and bias gradients as train_splits(rows, sms) partial
// sums over batch splits, each a full copy in the parameter layout (W_l at
// woff[l], b_l at boff[l]; np parameters, a multiple of 8): part[s * np + i].
// Every parameter of every split is written (no zeroing needed); summed in
// split order by train_reduce (into g) or by train_adam.  part holds
// train_part_elems(np) floats.
int train_splits(int64_t rows, int sms);
size_t train_part_elems(size_t np);
cudaError_t train_grads(TrainBufs b, int64_t rows, float *part, size_t np,
                        const size_t woff[kLayers], const size_t boff[kLayers], unsigned *err,
                        int sms, cudaStream_t s);
cudaError_t train_reduce(const float *part, int splits, size_t np, float *g, cudaStream_t s);
// Adam on the np parameters with the gradient summed from the partials and
// the step's learning rate and bias corrections from ctl; writes the bf16
// weights (wbf [out][in] per layer) and the packed training weights.  The
// transposed bf16 copy of the GEMM path is not written.
cudaError_t train_adam(float *w, const float *part, int splits, float *m, float *v,
                       __nv_bfloat16 *wbf, __nv_bfloat16 *wtp, const size_t woff[kLayers],
                       size_t np, const StepCtl *ctl, float b1, float b2, float eps,
                       cudaStream_t s);

} // namespace mlp
} // namespace kerr
