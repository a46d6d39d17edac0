/*
 * lmunet.h -- C ABI of the learned warm start: a small 3-D U-Net that
 * predicts an initial half-resolution displacement for the LM optimizer of
 * lmreg.h, trained on fields the optimizer itself produced.
 *
 * The paper has no network: the optimizer it describes starts from zero (or
 * from the coarser pyramid level, Section 2.1).  This warm start is an
 * addition on top of it.  Its architecture is this library's own:
 *
 *   input (F, M)                              2 ch, D x H x W
 *   e0 = a(c1(a(c0(input))))                 16 ch, full resolution
 *   e1 = a(c3(a(c2(pool(e0)))))              32 ch, 1/2
 *   e2 = a(c5(a(c4(pool(e1)))))              64 ch, 1/4
 *   e3 = a(c7(a(c6(pool(e2)))))             128 ch, 1/8
 *   d2 = a(c9(a(c8([up(e3), e2]))))          64 ch, 1/4
 *   d1 = a(c11(a(c10([up(d2), e1]))))        32 ch, 1/2
 *   out = c12(d1)                             3 ch, 1/2
 *
 * c_i: 3x3x3 cross-correlation, zero padding 1, with bias; a: leaky ReLU,
 * slope 0.2; pool: 2x2x2 mean; up: 2x2x2 nearest copy; [a, b]: channel
 * concatenation.  out is the displacement at half resolution in
 * half-resolution voxels, channels (x, y, z) as in lmreg.h fields.
 * Training minimises the mean squared error to a target field with Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master weights.
 *
 * Precision: activations, weights and activation gradients are bfloat16;
 * every convolution is an implicit GEMM on the tensor cores with FP32
 * accumulation; weight gradients, the loss and the optimizer state are FP32
 * (loss reduced in FP64).
 *
 * Packed host weight layout (lm_unet_create, lm_unet_get_weights,
 * lm_unet_get_grads): for c0 .. c12 in order, the weights as
 * [cout][cin][kz][ky][kx] followed by the bias [cout], FP32.
 *
 * Errors and ownership follow lmreg.h: 0 = LM_OK, negative codes, message
 * in lm_last_error(); the caller owns every pointer it passes.
 */
#ifndef LMUNET_H
#define LMUNET_H

#include "lmreg.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LM_UNET_LAYERS 13

typedef struct lm_unet lm_unet;

/* Layer shapes (cin[i], cout[i] for c0 .. c12; each array holds
 * LM_UNET_LAYERS ints) and the number of FP32 values of the packed weight
 * layout.  Any pointer may be NULL. */
LM_API int lm_unet_shapes(int *cin, int *cout, long long *nparams);

/* Create a network for inputs of D x H x W voxels (each a multiple of 8,
 * at most 512) with the given packed initial weights (host, FP32; copied).
 * Work is ordered on cuda_stream (NULL = default stream).  The network
 * allocates its activations, gradients and optimizer state on the device
 * (about 240 bytes per input voxel).  LM_EINVAL on bad sizes or NULL
 * weights; LM_ENOMEM on allocation failure. */
LM_API int lm_unet_create(lm_unet **net, int D, int H, int W,
                          const float *init_weights, void *cuda_stream);
LM_API void lm_unet_destroy(lm_unet *net);

/* Predicted displacement for one pair: fixed and moving as lm_volume
 * (D x H x W, FP32 or BF16 device data); u_half: device
 * [3][D/2][H/2][W/2] FP32 (written).  Asynchronous on the net's stream. */
LM_API int lm_unet_forward(lm_unet *net, const lm_volume *fixed,
                           const lm_volume *moving, float *u_half);

/* One Adam step on the mean MSE of n pairs: fixed[i], moving[i] as for
 * lm_unet_forward, targets[i] device [3][D/2][H/2][W/2] FP32.  lr: Adam
 * step size.  loss (host, may be NULL) receives the mean MSE of the batch
 * before the update.  Synchronises the stream when loss is not NULL. */
LM_API int lm_unet_train_step(lm_unet *net, int n, const lm_volume *fixed,
                              const lm_volume *moving,
                              const float *const *targets, float lr,
                              double *loss);

/* Copy the FP32 master weights, or the gradients of the last train step
 * (before the update, summed over the batch), to host memory in the packed
 * layout.  Synchronises. */
LM_API int lm_unet_get_weights(lm_unet *net, float *host);
LM_API int lm_unet_get_grads(lm_unet *net, float *host);

/* Tensors of the network's last pass, for inspection: the tests check
 * every layer against the oracle on the network's own stored inputs (the
 * paper has no network; this serves its parity checks).  Activations are
 * those of the last lm_unet_forward, or of the last pair of the last
 * training step; gradients are those of that pair's backward pass.  The
 * backward pass reuses its buffers, so only these gradients survive it:
 * DY<i>, the gradient of layer c<i>'s output after its activation mask
 * (the operand of its weight gradient), and DX<i>, the gradient of c<i>'s
 * input. */
enum {
    LM_UNET_X0, LM_UNET_E0A, LM_UNET_E0, LM_UNET_P0, LM_UNET_E1A, LM_UNET_E1,
    LM_UNET_P1, LM_UNET_E2A, LM_UNET_E2, LM_UNET_P2, LM_UNET_E3A, LM_UNET_E3,
    LM_UNET_CAT2, LM_UNET_D2A, LM_UNET_D2, LM_UNET_CAT1, LM_UNET_D1A,
    LM_UNET_D1, LM_UNET_OUT,
    LM_UNET_DY0, LM_UNET_DY1, LM_UNET_DY2, LM_UNET_DY3, LM_UNET_DY4,
    LM_UNET_DY5, LM_UNET_DY6, LM_UNET_DY12,
    LM_UNET_DX2, LM_UNET_DX4, LM_UNET_DX6, LM_UNET_DX8, LM_UNET_DX10,
    LM_UNET_NTENSORS
};
/* which: one of the LM_UNET_* tensors.  level (host, may be NULL): the
 * pyramid level l of the tensor (its sizes are D >> l, H >> l, W >> l);
 * channels (host, may be NULL): its stored channel count C (the head's
 * output and its gradient hold 16, the last 13 of them zero).  host: NULL
 * to query only, else room for (D >> l)(H >> l)(W >> l) C floats that
 * receive the tensor channels-last [z][y][x][c], bfloat16 values widened
 * exactly.  Synchronises the net's stream.  LM_EINVAL on a NULL net or an
 * unknown which. */
LM_API int lm_unet_get_tensor(lm_unet *net, int which, float *host,
                              int *level, int *channels);

/* Single 3x3x3 convolution, zero padding 1 (the kernels the network uses).
 * Activations are channels-last bfloat16: x [D][H][W][cin],
 * y [D][H][W][cout] FP32; w bfloat16 [cout][27][cin] with tap
 * t = 9 kz + 3 ky + kx; bias FP32 [cout] or NULL; act 1 = leaky ReLU 0.2.
 * cin must be 2 or a multiple of 16, cout a multiple of 16, D, H, W >= 1.
 * All pointers are device pointers.  Asynchronous on cuda_stream. */
LM_API int lm_conv3d_forward(int D, int H, int W, int cin, int cout,
                             const void *x, const void *w, const float *bias,
                             int act, float *y, void *cuda_stream);
/* Gradients of sum(dy * conv(x, w, b)): dx (bfloat16 [D][H][W][cin], may be
 * NULL; overwritten), dw (FP32 [cout][27][cin]) and db (FP32 [cout], may be
 * NULL) are ACCUMULATED into.  dy: bfloat16 [D][H][W][cout].  Same shape
 * rules as lm_conv3d_forward. */
LM_API int lm_conv3d_backward(int D, int H, int W, int cin, int cout,
                              const void *x, const void *w, const void *dy,
                              void *dx, float *dw, float *db,
                              void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LMUNET_H */
