/* Price surrogate: a multilayer perceptron fitted to SFFT prices.
 *
 * This is not part of the paper's method. The paper builds the pricing map
 * as a tensor network (Sec. 3); this network is a learned stand-in for
 * repeated queries inside a parameter box, with the SFFT pricer as its
 * fallback. The library never trains it implicitly: a caller drives the
 * steps below.
 *
 * Network (L linear layers, widths w_0 .. w_L, w_L = 1):
 *   h_0 = x,  z_l = W_l h_{l-1} + b_l,  h_l = GELU(z_l) (l < L),  y = z_L,
 *   GELU(z) = z Phi(z), Phi the standard normal CDF.
 *
 * Layout and ownership (all pointers are device memory the caller owns,
 * except where "host" is said):
 *   - W_l: w_l x w_{l-1}, row-major, stored as bfloat16 bit patterns
 *     (uint16); the products accumulate in float32.
 *   - b_l: w_l floats.
 *   - activations: batch x width, row-major floats.
 *   - a stream argument is a cudaStream_t (NULL: the legacy default stream);
 *     every call only enqueues work on it and returns.
 * Errors: SFFT_EINVAL for bad sizes or NULL pointers (nothing enqueued),
 * SFFT_ECUDA when a launch fails.
 */
#ifndef SFFT_MLP_H
#define SFFT_MLP_H

#include <stdint.h>

#include "sfft.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SFFT_MLP_MAX_LAYERS 8

/* Arithmetic of the products (sfft_mlp.mode):
 *   SFFT_MLP_TENSOR_CORES: fifth-generation tensor cores (tcgen05.mma,
 *     bfloat16 operands, float32 accumulation in tensor memory). The inputs
 *     enter as the bfloat16 pair hi + lo (hi = bf16(x), lo = bf16(x - hi),
 *     about 16 significant bits); every hidden activation h_l is rounded to
 *     the nearest bfloat16 (ties to even) before the next product, and the
 *     workspace keeps those rounded values, so the backward pass
 *     differentiates the network as evaluated (the rounding passes gradients
 *     through unchanged). GELU is evaluated there with Hastings' rational
 *     approximation of erf (Abramowitz & Stegun 7.1.26, absolute error at
 *     most 1.5e-7), far inside the bfloat16 rounding that follows. Needs n_layers >= 2, w_0 <= 8, hidden widths that
 *     are multiples of 16 in [16, 256], w_L = 1, and a 16-byte aligned
 *     workspace and packed weights (net->tc_weights, from sfft_mlp_pack)
 *     (else SFFT_EINVAL).
 *   SFFT_MLP_CUDA_CORES: float32 CUDA-core products with float32
 *     activations, any widths. */
#define SFFT_MLP_TENSOR_CORES 0
#define SFFT_MLP_CUDA_CORES 1

typedef struct sfft_mlp {
  int32_t n_layers;                          /* L, 1..SFFT_MLP_MAX_LAYERS */
  int32_t width[SFFT_MLP_MAX_LAYERS + 1];    /* w_0 .. w_L, each 1..1024; w_L = 1 */
  int32_t mode;                              /* SFFT_MLP_TENSOR_CORES or SFFT_MLP_CUDA_CORES */
  const uint16_t *w[SFFT_MLP_MAX_LAYERS];    /* W_l as bfloat16 bits */
  const float *b[SFFT_MLP_MAX_LAYERS];       /* b_l */
  const void *tc_weights;                    /* SFFT_MLP_TENSOR_CORES: the weights in the
                                                tensor cores' operand layout, written by
                                                sfft_mlp_pack (16-byte aligned); refresh
                                                it after every change of the W_l */
} sfft_mlp;

/* Bytes of the packed weight image of a network the tensor-core path takes
 * (-1 for any other shape). */
int64_t sfft_mlp_pack_bytes(const sfft_mlp *net);

/* Write the packed weight image of net's bfloat16 W_l into `packed` (device,
 * sfft_mlp_pack_bytes(net) bytes, 16-byte aligned): layer 1 as [W_1 | W_1]
 * (the weights of the hi and lo input halves), every later layer as K-chunks
 * of 64 in the K-major operand layout of the tensor cores, the output layer's
 * single row padded with zero rows to 16. */
sfft_status sfft_mlp_pack(const sfft_mlp *net, void *packed, void *stream);

/* Floats of the workspace that sfft_mlp_forward fills for a later
 * sfft_mlp_backward: z_l and h_l of every layer, batch rows each. */
int64_t sfft_mlp_workspace_floats(const sfft_mlp *net, int64_t batch);

/* Map raw query rows (raw: batch x n_in doubles, row-major) to network
 * inputs x = 2 (raw - lo) / (hi - lo) - 1 (floats, batch x n_in). lo, hi:
 * n_in doubles each, hi > lo. in_box[i] (may be NULL) is set to 1 when every
 * coordinate of row i lies in [lo, hi], else 0. */
sfft_status sfft_mlp_normalize(const double *raw, int64_t batch, int32_t n_in, const double *lo,
                               const double *hi, float *x, int32_t *in_box, void *stream);

/* Forward pass: y (batch floats) = network(x), in the arithmetic net->mode
 * names. Either ws holds
 * sfft_mlp_workspace_floats(net, batch) floats, which keep z_l and h_l of
 * every layer for sfft_mlp_backward, or ws is NULL and ws_scratch holds
 * 2 * batch * max(w_1 .. w_{L-1}) floats used as two ping-pong activation
 * buffers (inference). */
sfft_status sfft_mlp_forward(const sfft_mlp *net, const float *x, int64_t batch, float *y, float *ws,
                             float *ws_scratch, void *stream);

/* Number of tensor-core forward launches whose bounded waits on the tensor
 * cores expired since the library was loaded (their outputs are not valid);
 * 0 in a healthy run. Synchronises the device. */
int32_t sfft_mlp_tc_timeouts(void);

/* Mean squared error of y against t (batch floats each): dy = 2 (y - t) /
 * batch, and *loss (device float, may be NULL) = mean (y - t)^2. */
sfft_status sfft_mlp_mse_grad(const float *y, const float *t, int64_t batch, float *dy, float *loss,
                              void *stream);

/* Backward pass after a forward pass that filled ws: gradients of the loss
 * whose derivative with respect to y is dy. gw[l] (w_l x w_{l-1} floats) and
 * gb[l] (w_l floats) are overwritten. scratch: 2 * batch * max(width)
 * floats. */
sfft_status sfft_mlp_backward(const sfft_mlp *net, const float *x, int64_t batch, const float *ws,
                              const float *dy, float *const *gw, float *const *gb, float *scratch,
                              void *stream);

/* One Adam step (Kingma & Ba 2015, bias-corrected moments) on count
 * parameters: p (float master copy), m, v updated in place from g;
 * p_bf16 (may be NULL) receives p rounded to bfloat16 (nearest, ties to
 * even). step counts from 1. */
sfft_status sfft_mlp_adam(int64_t count, float *p, uint16_t *p_bf16, const float *g, float *m,
                          float *v, float lr, float beta1, float beta2, float eps, int64_t step,
                          void *stream);

#ifdef __cplusplus
}
#endif

#endif
