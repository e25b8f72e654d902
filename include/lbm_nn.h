/*
 * lbm_nn.h -- C ABI of the layer kernels of the learned surrogate: a small
 * convolutional U-Net that maps the moment fields U(t) of a periodic lattice to
 * U(t + k dt), trained on trajectories of the lattice Boltzmann solver itself.
 * The paper has no such component; these calls serve the library's surrogate.
 *
 * Conventions
 *   - Activations: FP32, channels-last [B][H][W][C], device memory.  H and W are
 *     powers of two; every convolution pads circularly (periodic lattices).
 *   - Weights: BF16 (stored as 16-bit words) [Cout][KS][KS][Cin], KS in {1, 3};
 *     biases FP32 [Cout].  FP32 master weights live with the optimiser.
 *   - Convolutions run on the tensor cores (BF16 inputs, FP32 accumulation) with
 *     activations split into two BF16 halves, so the BF16 weights are the only
 *     rounding of the forward pass.  3x3 convolutions with H >= 16, W >= 8 and
 *     Cout a multiple of 32 use tcgen05.mma with the accumulator in tensor
 *     memory; other sizes (and LBM_NN_MMA_SYNC) use mma.sync kernels.
 *   - Two-input convolutions read the channel concatenation [x1 | x2]; two-output
 *     ones write channels [0, Co1) to y1 and [Co1, Cout) to y2.  LBM_NN_ACCUMULATE
 *     adds the result into the destination instead of overwriting it.
 *   - Channel counts: C1, C2 multiples of 32 (C2 may be 0); Cout a multiple of 8.
 *   - All calls are asynchronous on `stream` (NULL = legacy stream) and return
 *     LBM_ERR_ARG for invalid sizes or NULL pointers, LBM_ERR_CUDA if a launch
 *     failed.  The caller owns every buffer.
 */
#ifndef LBM_NN_H
#define LBM_NN_H

#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Flags of the convolution calls. */
enum {
    LBM_NN_RELU = 1,        /* apply max(0, .) to the output (forward) */
    LBM_NN_ACCUMULATE = 2,  /* add the result into the destination instead of overwriting it */
    LBM_NN_X1_HALF = 4,     /* x1 is stored at (H/2, W/2) and read nearest-upsampled to (H, W) */
    LBM_NN_ACT_BF16 = 8,    /* forward: activations as one BF16 value instead of the hi/lo pair
                               (half the tensor-core work; activations rounded to BF16) */
    LBM_NN_MMA_SYNC = 16,   /* forward: use the mma.sync kernels even where the tcgen05 kernel applies
                               (same arithmetic, other summation order) */
    LBM_NN_WGRAD_PER_TAP = 32 /* weight gradient: the per-tap kernel even where the block-tiled 3x3
                                 kernel applies (same products, other summation order) */
};

/* y = act(conv_KS(x, w) + bias), act = ReLU with LBM_NN_RELU; flags as above (any other
 * bit returns LBM_ERR_ARG). */
lbm_status lbm_nn_conv_forward(const float* x1, int32_t C1, const float* x2, int32_t C2, const void* w_bf16,
                               const float* bias, float* y1, int32_t Co1, float* y2, int32_t Cout, int32_t B,
                               int32_t H, int32_t W, int32_t KS, int32_t flags, void* stream);

/* Launch counters since the library was loaded (host side; out must hold four values):
 * forward convolutions on the tcgen05 kernel (out[0]) and on the mma.sync kernels (out[1]);
 * weight gradients on the block-tiled 3x3 kernel (out[2]) and on the per-tap kernel (out[3]). */
lbm_status lbm_nn_conv_counts(int64_t* out);

/* Synchronises `stream`; LBM_ERR_TIMEOUT if a bounded wait inside a tcgen05 convolution ran
 * out since the last call (the output of that convolution is invalid; the flag is cleared),
 * LBM_ERR_CUDA if a launch or the stream failed, else LBM_OK. */
lbm_status lbm_nn_check(void* stream);

/* Workspace bytes lbm_nn_conv_backward_weight needs for these sizes (Cin = C1 + C2). */
int64_t lbm_nn_wgrad_workspace_bytes(int32_t Cin, int32_t Cout, int32_t B, int32_t H, int32_t W, int32_t KS);

/* dw[co][ky][kx][ci] (+)= sum over pixels of dy[p][co] * x[p + (ky, kx) - KS/2][ci]; FP32 output,
 * reduced over pixel splits in a fixed order (deterministic).  3x3 with H, W >= 16 and Cout a
 * multiple of 32 runs on 16x16-pixel blocks with all nine taps per CTA; other sizes (and
 * LBM_NN_WGRAD_PER_TAP) one tap per CTA.  flags: LBM_NN_ACCUMULATE, LBM_NN_X1_HALF,
 * LBM_NN_WGRAD_PER_TAP (others return LBM_ERR_ARG). */
lbm_status lbm_nn_conv_backward_weight(const float* dy, int32_t Cout, const float* x1, int32_t C1, const float* x2,
                                       int32_t C2, int32_t B, int32_t H, int32_t W, int32_t KS, float* dw,
                                       int32_t flags, void* workspace, int64_t workspace_bytes, void* stream);

/* Workspace (device bytes) lbm_nn_bias_grad needs for P pixels and C channels. */
int64_t lbm_nn_bias_grad_workspace_bytes(int64_t P, int32_t C);

/* db[c] = sum over P pixels of dy[p][c] (dy: [P][C] FP32, device).  Two passes in a
 * fixed order (per-block partials in `workspace`, then their sum), so results are
 * reproducible.  workspace_bytes below lbm_nn_bias_grad_workspace_bytes(P, C), null
 * pointers or P, C <= 0 return LBM_ERR_ARG. */
lbm_status lbm_nn_bias_grad(const float* dy, int64_t P, int32_t C, float* db, void* workspace,
                            int64_t workspace_bytes, void* stream);

/* wt[ci][KS*KS-1-tap][co] = w[co][tap][ci]: with it, lbm_nn_conv_forward of dy gives the data gradient. */
lbm_status lbm_nn_weight_flip(const void* w_bf16, int32_t Cout, int32_t Cin, int32_t KS, void* wt_bf16, void* stream);

/* dy[i] = 0 where y[i] <= 0 (y = ReLU output). */
lbm_status lbm_nn_relu_backward(float* dy, const float* y, int64_t n, void* stream);

/* 2x2 average pooling [B][H][W][C] -> [B][H/2][W/2][C] and its gradient. */
lbm_status lbm_nn_pool(const float* x, int32_t B, int32_t H, int32_t W, int32_t C, float* y, void* stream);
lbm_status lbm_nn_pool_backward(const float* dy, int32_t B, int32_t H, int32_t W, int32_t C, float* dx, int32_t beta,
                                void* stream);

/* nearest-neighbour 2x upsampling [B][H][W][C] -> [B][2H][2W][C] and its gradient. */
lbm_status lbm_nn_upsample(const float* x, int32_t B, int32_t H, int32_t W, int32_t C, float* y, void* stream);
lbm_status lbm_nn_upsample_backward(const float* dy, int32_t B, int32_t H, int32_t W, int32_t C, float* dx,
                                    int32_t beta, void* stream);

/* loss_out (device, FP64) = sum over P pixels and the first cvalid channels of (out - tgt)^2;
 * dout (optional) = 2 (out - tgt) * grad_scale on those channels, 0 elsewhere.
 * workspace: 512 doubles of device memory. */
lbm_status lbm_nn_mse(const float* out, const float* tgt, int64_t P, int32_t C, int32_t cvalid, float grad_scale,
                      float* dout, double* workspace, double* loss_out, void* stream);

/* Adam step `step` (>= 1) on FP32 master weights w with gradient g and moments m, v;
 * writes the BF16 working copy when w_bf16 is not NULL. */
lbm_status lbm_nn_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                       float eps, int64_t step, void* w_bf16, void* stream);

/* y = bf16(x) (round to nearest even). */
lbm_status lbm_nn_to_bf16(const float* x, int64_t n, void* y_bf16, void* stream);

/* Network input: channel c < nf is U[b][c] / scale[c] (U FP64, sample b at U + b*sample_stride,
 * fields [nf][H][W]); channel nf is extra[b] when extra != NULL; the rest are zero. */
lbm_status lbm_nn_pack_input(const double* U, int64_t sample_stride, int32_t nf, const double* scale,
                             const float* extra, int32_t B, int32_t H, int32_t W, int32_t C, float* x, void* stream);

/* Training target t[b][y][x][c] = (Unext - Unow)[b][c][y][x] / scale[c] for c < nf, 0 otherwise. */
lbm_status lbm_nn_pack_target(const double* Unow, const double* Unext, int64_t sample_stride, int32_t nf,
                              const double* scale, int32_t B, int32_t H, int32_t W, int32_t C, float* t, void* stream);

/* Prediction Uout[b][c] = Uin[b][c] + scale[c] * net[b][.][.][c], c < nf (FP64 fields). */
lbm_status lbm_nn_residual_output(const double* Uin, int64_t in_stride, const float* net, int32_t C,
                                  const double* scale, int32_t nf, int32_t B, int32_t H, int32_t W, double* Uout,
                                  int64_t out_stride, void* stream);

/* Periodic second-order central differences of FP64 fields (spacing dx): the
 * derivatives the re-initialisation (Eq. ic_second) needs after a surrogate jump. */
lbm_status lbm_nn_gradient(const double* U, int64_t sample_stride, int32_t nf, int32_t B, int32_t H, int32_t W,
                           double dx, double* dUx, double* dUy, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_NN_H */
