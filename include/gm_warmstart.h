/*
 * gm_warmstart.h -- C ABI of the learned warm start for the Tikhonov CGLS
 * inversion of gravity data.
 *
 * The paper computes the forward and transpose products (Sec. 3) and names
 * their use inside an inversion as the application it enables (Sec. 1 and
 * Sec. 6); it has no network.  This library adds one: a convolutional network
 * net(d) that maps a data grid d[S][S] (stations sx = sy = S, gravity, no
 * padding) to a model m[16][S][S] of the same grid (16 depth layers), trained
 * on (model, G model + noise) pairs made with the forward product.  Its
 * prediction is the starting point x0 of gm_cgls; CGLS from x0 = 0 stays the
 * fallback and the yardstick of its error.
 *
 * Architecture (tensors N x C x D x H x W, x fastest; every convolution has
 * kernel 3 in each convolved axis, "same" zero padding and a bias):
 *   encoder  E0  conv 1x3x3, 1 -> 32 channels, stride 1, ReLU         (S x S)
 *            E1..E4 conv 1x3x3, stride (1,2,2): 32 -> 64 -> 128 -> 256
 *            -> 512 channels, ReLU                             (down to S/16)
 *   reshape  512 x 1 x S/16 x S/16 read as 128 x 4 x S/16 x S/16
 *            (channel c' and depth z of the new tensor are channel 4 c' + z)
 *   decoder  D1 nearest up-sampling (2,2,2), conv 3x3x3 128 -> 64, ReLU
 *            D2 up (2,2,2), conv 3x3x3 64 -> 32, ReLU
 *            D3 up (1,2,2), conv 3x3x3 32 -> 16, ReLU
 *            D4 up (1,2,2), conv 3x3x3 16 -> 1, linear        (16 x S x S)
 *   scaling  net(d) = out_scale * f(in_scale * d)
 * Parameters (1,858,849 for any S): for each layer in the order above its
 * weights w[co][ci][kd][kh][kw] followed by its biases b[co], one flat FP32
 * vector.  Every convolution of the forward pass and of the backward pass
 * (data and weight gradients) is a tensor-core GEMM with BF16 operands and
 * FP32 accumulation: BF16 copies of the weights, and activations / gradients
 * (stored in FP32) rounded to BF16 as they are gathered; bias gradients are
 * sums of the BF16-rounded output gradients.  Adam updates the FP32 master
 * weights and refreshes the BF16 copies.
 *
 * Layouts: d[n][y][x] (batch n < batch, S x S, float), m[n][z][y][x] (16 x S x
 * S, float), both contiguous device buffers owned by the caller.  The handle
 * owns the weights, Adam moments and every activation / gradient buffer,
 * sized for max_batch at creation.  Calls are ordered on the CUDA stream
 * passed in (NULL = legacy default stream); calls on one handle must not
 * overlap in time.  Errors: a gm_status, with a message in
 * gm_net_last_error(); bad arguments never reach the device.
 */
#ifndef GM_WARMSTART_H
#define GM_WARMSTART_H

#include "gravmag.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gm_net *gm_net_handle;

/* A network for S x S data (S a multiple of 16, 16 <= S <= 1024) and depth 16,
 * with buffers for up to max_batch examples (max_batch * 16 * S^2 <= 2^30).  Weights: He-uniform from a
 * counter-based generator (splitmix64 of seed and the parameter index);
 * biases 0.  NULL on failure (gm_net_last_error says why). */
GM_API gm_net_handle gm_net_create(int grid, int depth, int max_batch, unsigned long long seed);
GM_API gm_status gm_net_destroy(gm_net_handle net);
GM_API int64_t gm_net_num_params(gm_net_handle net);

/* net(d) = out_scale * f(in_scale * d); both > 0 (defaults 1). */
GM_API gm_status gm_net_set_scales(gm_net_handle net, float in_scale, float out_scale);

/* m_dev[batch][16][S][S] = net(d_dev[batch][S][S]). */
GM_API gm_status gm_net_forward(gm_net_handle net, const float *d_dev, float *m_dev, int batch, void *stream);

/* One training step on a batch: the loss
 *   L = 1/(batch 16 S S) SUM (f(in_scale d) - m / out_scale)^2,
 * its gradient with respect to every parameter (left in the gradient buffer,
 * readable with gm_net_get_params(..., 1)), and, when lr > 0, one Adam step
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).  d_dev[count][S][S] and
 * m_dev[count][16][S][S] hold `count` examples; the batch is examples
 * index_dev[0..batch-1] (a device int32 array) or, with index_dev = NULL,
 * examples 0..batch-1 (then batch <= count).  An index outside [0, count)
 * reads nothing: that example is zeros and the next call that synchronises
 * returns GM_EINVAL.  loss_host (may be NULL) receives L (plus lambda times
 * the data term, see gm_net_set_data_term); the call then synchronises the
 * stream and reports a bad index. */
GM_API gm_status gm_net_train_step(gm_net_handle net, const float *d_dev, const float *m_dev, int count,
                                   const int32_t *index_dev, int batch, float lr, float *loss_host, void *stream);

/* Data-consistency term of the training loss: with lambda > 0 every
 * gm_net_train_step adds
 *   lambda * 1/(batch S S) SUM (in_scale (G m_pred - d))^2,   m_pred = net(d),
 * and its gradient 2 lambda/(batch S S) in_scale out_scale G^T r (r the
 * scaled misfit) with respect to f, computed with apply_forward and
 * apply_transpose of `op` (one each per example, on the train step's stream).
 * op must be an FP32 handle with sx = sy = nx = ny = S (no padding) and
 * nz = 16; it is not owned and must outlive its use.  lambda = 0 removes the
 * term.  Allocates the term's buffers on first use. */
GM_API gm_status gm_net_set_data_term(gm_net_handle net, gm_handle op, float lambda);

/* Model and data terms of the last train step that returned its loss. */
GM_API gm_status gm_net_last_losses(gm_net_handle net, float *model_term, float *data_term);

/* Copy a parameter-sized FP32 vector to / from the host: which = 0 weights
 * (master copy; setting it refreshes the BF16 copy), 1 last gradient (get
 * only), 2 Adam first moment, 3 Adam second moment.  n must equal
 * gm_net_num_params.  Synchronous. */
GM_API gm_status gm_net_get_params(gm_net_handle net, float *host, int64_t n, int which);
GM_API gm_status gm_net_set_params(gm_net_handle net, const float *host, int64_t n, int which);
GM_API gm_status gm_net_get_step(gm_net_handle net, int64_t *step);
GM_API gm_status gm_net_set_step(gm_net_handle net, int64_t step);

/* One convolution of the network's kind on its own, through the same
 * tensor-core kernels (BF16 operands, FP32 accumulation): a 3-D
 * cross-correlation with kernel KD x 3 x 3 (KD = 1 or 3), in-plane stride 1
 * or 2, "same" zero padding (KD/2, 1, 1), on x[N][CI][ID][IH][IW]; the output
 * is [N][CO][ID][OH][OW] with OH = (IH-1)/stride + 1, OW likewise.  CI and CO
 * are powers of two (<= 4096).  w[CO][CI][KD][3][3] (device, FP32) is rounded
 * to BF16 inside.
 *   mode 0: out = conv(x) + b  (b may be NULL; g unused)
 *   mode 1: out[N][CI][ID][IH][IW] = the data gradient for the output
 *           gradient g[N][CO][ID][OH][OW]  (x unused)
 *   mode 2: out[CO][CI][KD][3][3] = the weight gradient for x and g;
 *           bias_grad[CO] (may be NULL) = SUM over n and positions of g
 * Operands are rounded to BF16 as the network's kernels round them.  All
 * pointers are device pointers owned by the caller; the call allocates
 * scratch, runs on `stream` and synchronises it. */
GM_API gm_status gm_conv3d(int mode, int N, int CI, int CO, int ID, int IH, int IW, int KD, int stride,
                           const float *x, const float *g, const float *w, const float *b, float *out,
                           float *bias_grad, void *stream);

/* Kernels launched by the last forward / train-step call on this handle. */
GM_API int gm_net_last_launch_count(gm_net_handle net);
/* Message of the last failing gm_net_* call of this thread. */
GM_API const char *gm_net_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GM_WARMSTART_H */
