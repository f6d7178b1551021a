// Tensor-core (tcgen05) kernels of the learned inverse: inference
// (conv_tc.cu) and the training step's convolution backward (train_tc.cu).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pchase.h"

namespace pchase {

// Inference of the first two layers in one kernel: out [nb][128][64] BF16 =
// layer 2's GELU outputs for x [nb][512] FP32 (rounded to BF16 as inputs),
// W1 [64][5] BF16 + bias1, W2 [64][5*64] BF16 + bias2.  The first layer's
// outputs never leave the SM.  A wait that gives up ORs PCHASE_DEV_TIMEOUT
// into *status (device).
cudaError_t conv12_tc(const float *x, int nb, const __nv_bfloat16 *W1, const float *bias1,
                      const __nv_bfloat16 *W2, const float *bias2, __nv_bfloat16 *out,
                      uint32_t *status, int sms, cudaStream_t st);

// Inference of layers 3 and 4 in one kernel: out [nb][32][64] BF16 = layer
// 4's GELU outputs for x [nb][128][64] BF16 (layer 2's), W3, W4 [64][5*64]
// BF16 + bias3, bias4.  Layer 3's outputs never leave the SM.  A wait that
// gives up ORs PCHASE_DEV_TIMEOUT into *status (device).
cudaError_t conv34_tc(const __nv_bfloat16 *x, int nb, const __nv_bfloat16 *W3, const float *bias3,
                      const __nv_bfloat16 *W4, const float *bias4, __nv_bfloat16 *out,
                      uint32_t *status, int sms, cudaStream_t st);

// logits [nb][31] FP32 = heads(GELU(FC(act))) for act [nb][2048] BF16 (the
// flattened last convolution), W4 [256][2048] BF16 + bias4, W5 [31][256] BF16
// + bias5; hidden activations rounded to BF16 as the heads' operands.  FC and
// heads both run on tcgen05 tensor cores, all 256 hidden units of a 128-row
// tile in one CTA; each logit has one writer.  A wait that gives up ORs
// PCHASE_DEV_TIMEOUT into *status.
cudaError_t fc_heads_tc(const __nv_bfloat16 *act, int nb, const __nv_bfloat16 *W4,
                        const float *bias4, const __nv_bfloat16 *W5, const float *bias5,
                        float *logits, uint32_t *status, cudaStream_t st);

// Training step, forward of one 64-channel convolution layer (lout = 128, 64
// or 32; lin = 2 lout): pre [nb * lout][64] FP32 = the pre-activations for x
// [nb][lin][64] BF16, W [64][5*64] BF16 + bias; out [nb * lout][64] BF16 =
// GELU(pre) with the exact tanh.  tcgen05 tensor cores; a wait that gives up
// ORs PCHASE_DEV_TIMEOUT into *status (device).
cudaError_t conv_fwd_tc(const __nv_bfloat16 *x, int nb, int lout, const __nv_bfloat16 *W,
                        const float *bias, float *pre, __nv_bfloat16 *out, uint32_t *status, int sms,
                        cudaStream_t st);

// Training step, backward of one 64-channel convolution layer (lout = 128,
// 64 or 32 output positions per trace; lin = 2 lout): given dact [nb * lout][64]
// FP32 (gradient of the layer's GELU outputs), pre [nb * lout][64] FP32 (its
// pre-activations), x [nb][lin][64] BF16 (its inputs) and W [64][5*64] BF16,
// adds the weight gradient into gW [64][5*64] and the bias gradient into
// gb [64] (FP32 atomics: both must hold their running sums, usually zero),
// and writes the input gradient dx [nb][lin][64] FP32.  tcgen05 tensor cores;
// a wait that gives up ORs PCHASE_DEV_TIMEOUT into *status (device).
cudaError_t conv_back_tc(const float *dact, const float *pre, const __nv_bfloat16 *x, int nb,
                         int lout, const __nv_bfloat16 *W, float *gW, float *gb, float *dx,
                         uint32_t *status, int sms, cudaStream_t st);

// The same for the first layer (one input channel, x [nb][512] BF16, W
// [64][5]; no input gradient), on CUDA cores.
cudaError_t conv0_back(const float *dact, const float *pre, const __nv_bfloat16 *x, int nb,
                       float *gW, float *gb, int sms, cudaStream_t st);

// C = A B^T on the tcgen05 tensor cores: A [M][K], B [N][K] BF16 with row
// strides lda, ldb (multiples of 8 elements, 16-byte aligned bases).  Tiles of
// 128 x bn (bn = 32 or 128; 64 for the GELU form); K split into k_slices
// slices.  Without pre: C[m * ldc + n] (C[n * ldc + m] when transposed)
// = sum + bias[n] (bias optional), FP32 atomics when atomic (required for
// k_slices > 1).  With pre (bn = 64, one slice): pre[m * ldc + n] = sum + bias[n]
// and Cb[m * ldc + n] = BF16(GELU(that)).  A wait that gives up ORs
// PCHASE_DEV_TIMEOUT into *status.
cudaError_t tc_gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N,
                    int K, int bn, int k_slices, const float *bias, float *C, int ldc, bool atomic,
                    bool transposed, float *pre, __nv_bfloat16 *Cb, uint32_t *status,
                    cudaStream_t st);

// out [Cpad][ldo] = transpose of in [R][C] (row stride ldi), zero beyond R
// columns and C rows.
cudaError_t transpose_bf16(const __nv_bfloat16 *in, int R, int C, int ldi, __nv_bfloat16 *out,
                           int ldo, int Cpad, cudaStream_t st);

}  // namespace pchase
