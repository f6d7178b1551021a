// Tensor-core (tcgen05) convolution of the learned inverse (conv_tc.cu).
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

}  // namespace pchase
