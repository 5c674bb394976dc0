/*
 * unet.h — C ABI of the learned inlet-profile initialiser: a 4-level U-Net
 * that maps an observed steady velocity field and the obstacle mask to a first
 * guess of the inlet density profile, from which the gradient inversion of
 * lbm.h starts.  The paper proposes such a network as future work (closing
 * remarks of section 3 and section 4); it has no architecture or training
 * recipe, so this one is ours:
 *
 *   input   x[b][h][w][C0] bf16 (NHWC): u_x * s, u_y * s, mask, zeros (C0 = 8)
 *   level l (l = 0..3, c_l = base 2^l): two 3x3 convolutions (zero padding) +
 *           ReLU; 2x2 max-pool between encoder levels
 *   decoder (l = 2..0): 2x2 stride-2 transposed convolution c_{l+1} -> c_l,
 *           concatenation [upsampled, skip], two 3x3 convolutions + ReLU
 *   head    1x1 convolution c_0 -> 1 and the mean over w: out[b][h], the inlet
 *           profile (rho_in - rho_out) / 1e-3 of row h
 *   loss    mean over b, h of (out - target)^2
 *
 * Weights are FP32 master copies (one flat vector, the order of
 * unet_param_layout) converted to BF16 operand layouts by
 * unet_prepare_weights; activations are BF16; every product accumulates in
 * FP32 on the tensor cores (tcgen05.mma with TMEM accumulators, or mma.sync
 * m16n8k16: unet_set_engine).  Gradients of the weights are FP32.
 *
 * Conventions as in lbm.h: every call returns an lbm_status, is asynchronous
 * on the given stream (a cudaStream_t as void*), and the caller owns every
 * device buffer.  Sizes: height and width multiples of 8, base a multiple of 8.
 */
#ifndef UNET_H
#define UNET_H

#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct unet_desc {
    int32_t base;    /* channels of level 0 (multiple of 8, >= 8); level l has base * 2^l */
    int32_t height;  /* rows h (the inlet profile length), multiple of 8 */
    int32_t width;   /* columns w, multiple of 8 */
    int32_t batch;   /* samples per forward / backward call, >= 1 */
} unet_desc;

#define UNET_IN_CHANNELS 8

/* The GEMM engine of the convolutions (process-wide).  UNET_ENGINE_TCGEN05
 * (default): the 3x3 convolutions, their input gradients and the transposed
 * convolutions' forward products run on the Blackwell tensor cores
 * (tcgen05.mma, BF16 operands staged by TMA in shared memory, FP32
 * accumulator in tensor memory) where the level's width is a multiple of 16,
 * its height of 8, the gathered channel count 32 or a multiple of 64 and the
 * output channel count a multiple of 32; the other products, and every
 * product with UNET_ENGINE_MMA_SYNC, run the mma.sync kernel.  Both engines
 * accumulate in FP32 over the same terms (in different orders).
 * Errors: INVALID_ARG for an unknown engine. */
enum { UNET_ENGINE_MMA_SYNC = 0, UNET_ENGINE_TCGEN05 = 1 };
LBM_API lbm_status unet_set_engine(int32_t engine);

/* LBM_OK, or LBM_ERR_TIMEOUT if a bounded wait of a tensor-core kernel gave
 * up since the last call (the kernel then skipped its output); clears the
 * flag.  Synchronises the device. */
LBM_API lbm_status unet_get_status(void);

/* Number of FP32 parameters, and the offset and element count of parameter
 * tensor i (i = 0..n_tensors-1, the order: enc0a.w, enc0a.b, enc0b.w, enc0b.b,
 * ..., enc3b.b, up2.w, up2.b, dec2a.w, dec2a.b, dec2b.w, dec2b.b, up1..., dec0b.b,
 * head.w, head.b; a 3x3 weight is [3][3][c_in][c_out], a transposed-convolution
 * weight [2][2][c_in][c_out], the head weight [c_0]). */
LBM_API lbm_status unet_param_layout(int32_t base, int32_t* n_tensors, int64_t* n_params, int64_t* offsets,
                                     int64_t* counts);

/* Device workspace for one descriptor: BF16 weight layouts, activations,
 * their gradients, argmax indices, split-K partials.  Errors: INVALID_ARG. */
LBM_API lbm_status unet_workspace_size(const unet_desc* d, size_t* bytes);

/* Input packing: x[b][h][w][c] = (u_x s, u_y s, mask, 0...) from the velocity
 * fields d_u (double [batch][2][h][w], as lbm_macroscopic writes them) and the
 * masks d_mask (uint8 [batch][h][w], nonzero = solid).  d_x is bf16 (uint16). */
LBM_API lbm_status unet_pack_input(const unet_desc* d, const double* d_u, const uint8_t* d_mask, double scale,
                                   uint16_t* d_x, void* stream);

/* FP32 master weights -> the BF16 operand layouts in the workspace. */
LBM_API lbm_status unet_prepare_weights(const unet_desc* d, const float* d_params, void* d_ws, void* stream);

/* Forward pass of d_x (bf16 [batch][h][w][8]) -> d_out (float [batch][h]);
 * keeps the activations in d_ws for unet_backward. */
LBM_API lbm_status unet_forward(const unet_desc* d, const uint16_t* d_x, float* d_out, void* d_ws, void* stream);

/* Loss against d_target (float [batch][h]) of the last forward of d_x (the
 * same input, still unchanged), into d_loss (float[1]), and the FP32 gradient
 * of every parameter into d_grad (the layout of unet_param_layout;
 * overwritten). */
LBM_API lbm_status unet_backward(const unet_desc* d, const uint16_t* d_x, const float* d_target, float* d_loss,
                                 float* d_grad, void* d_ws, void* stream);

/* Adam on the FP32 master weights (t 1-based). */
LBM_API lbm_status unet_adam(int64_t n, float* d_params, float* d_m, float* d_v, const float* d_grad, int32_t t,
                             float lr, float beta1, float beta2, float eps, void* stream);

#ifdef __cplusplus
}
#endif

#endif
