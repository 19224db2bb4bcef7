/* ccnet.h - C ABI of the learned initial guess: a small 3-D U-Net whose
 * convolutions are BF16 implicit-GEMM kernels on the fifth-generation tensor
 * cores (tcgen05, FP32 accumulation in tensor memory), trained on the GPU on
 * (f, volume fraction, boundary data) -> phi pairs that the multigrid solver
 * generates, and used as the starting guess of Alg. Multigrid.  The paper has
 * no learned component: the solve that follows the guess is the paper's
 * V-cycle iteration, which always finishes to the tolerance.
 *
 * Network (fixed): input 3 channels (stored as 16, the extra ones zero);
 * encoder levels l = 0..3 with 16 * 2^l channels, two 3x3x3 convolutions
 * (zero padding, bias, ReLU) per level and 2x2x2 average pooling between
 * levels; decoder levels l = 2..0: nearest-neighbour upsampling by 2 of level
 * l+1, concatenation with the encoder's level-l output, two 3x3x3
 * convolutions with ReLU; a 1x1x1 convolution to one output channel (FP32, no
 * activation).  1 460 449 parameters counted without the padded input
 * channels.  Grids n^3 with n a multiple of 8.
 *
 * Layouts.  Activations are NDHWC: a grid of n^3 cells (index (i*n + j)*n + k,
 * k fastest, as the solver's grid arrays) with the channels innermost, BF16.
 * A 3x3x3 weight tensor is [C_out][27][C_in] BF16 with tap t = (a*3 + b)*3 + c
 * for the offset (a-1, b-1, c-1) along (i, j, k); biases are FP32 [C_out].
 * All pointers are device pointers on the network's device unless stated;
 * the caller owns every buffer it passes.  Every call returns a cc_status
 * (include/ccmg.h) and never aborts; calls on one network are not thread-safe.
 */
#ifndef CCNET_H
#define CCNET_H

#include <stdint.h>

#include "ccmg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* struct ccnet is declared in ccmg.h */

/* One 3x3x3 convolution layer on the tensor cores (building block, tested on
 * its own against a CPU direct convolution):
 *   y[v][co] = act(b[co] + sum_t sum_ci w[co][t][ci] * x[v + off(t)][ci])
 * over an n^3 grid with zero padding; x has cin channels, y cout.  cin and
 * cout are multiples of 16 with cin <= 256 and cout <= 256.  relu != 0 applies
 * max(0, .).  b may be NULL (no bias).  y_bf16 receives BF16 output, y_f32 (may
 * be NULL) also the FP32 value before rounding.  Errors: CC_ERR_INVALID_ARG
 * for bad sizes or NULL x/w/y_bf16; CC_ERR_TIMEOUT if a bounded wait on the
 * tensor cores ran out (the kernel then stops and frees its tensor memory). */
cc_status ccnet_conv3d(int device, int n, int cin, int cout, const uint16_t* x, const uint16_t* w, const float* b,
                       int relu, uint16_t* y_bf16, float* y_f32, void* stream);

/* Backward of one layer (given g = dL/dy already multiplied by the ReLU
 * derivative, BF16 [n^3][cout]):
 *   dx[v][ci] = sum_t sum_co w[co][t][ci] * g[v - off(t)][co]   (FP32 out, may be NULL)
 *   dw[co][t][ci] += sum_v g[v][co] * x[v + off(t)][ci]         (FP32, accumulated)
 *   db[co] += sum_v g[v][co]                                   (FP32, may be NULL)
 * dx runs on the tensor cores as a convolution with the taps mirrored and the
 * channel roles swapped; dw as a GEMM over the grid (K = n^3) per tap, whose
 * 128-row tile holds cout <= 128 (CC_ERR_INVALID_ARG otherwise). */
cc_status ccnet_conv3d_backward(int device, int n, int cin, int cout, const uint16_t* x, const uint16_t* w,
                                const uint16_t* g, float* dx, float* dw, float* db, void* stream);

/* The network.  ccnet_create allocates parameters (seeded He initialisation),
 * Adam moments and the work buffers for grids up to n_max^3 on `device`. */
cc_status ccnet_create(int device, int n_max, uint64_t seed, ccnet** out);
void ccnet_destroy(ccnet* net);
/* Number of parameters (FP32 master copies) and host copies of them, in a
 * fixed order (per layer: weights [C_out][27][C_in_real] then biases). */
cc_status ccnet_num_params(const ccnet* net, long long* count);
cc_status ccnet_get_params(const ccnet* net, float* host);
cc_status ccnet_set_params(ccnet* net, const float* host);

/* Forward pass on an n^3 grid: input FP32 [n^3][3] (host or device per
 * `where`, CC_HOST/CC_DEVICE), output FP32 phi guess [n^3] (same side). */
cc_status ccnet_forward(ccnet* net, int n, const float* input, float* out, int where);

/* One training step on a batch of `batch` grids of n^3 cells (inputs [batch][n^3][3],
 * targets [batch][n^3], weights [batch][n^3] (0 outside the domain), device
 * FP32): mean weighted squared error, backward through every layer, Adam
 * (lr, beta1 0.9, beta2 0.999, eps 1e-8).  *loss receives the batch loss
 * (host).  Gradients are also left in the network (ccnet_get_grads). */
cc_status ccnet_train_step(ccnet* net, int n, int batch, const float* inputs, const float* targets,
                           const float* weights, float lr, float* loss);
/* Loss and gradients only (no update), for gradient checks. */
cc_status ccnet_loss_grad(ccnet* net, int n, int batch, const float* inputs, const float* targets,
                          const float* weights, float* loss);
cc_status ccnet_get_grads(const ccnet* net, float* host);

#ifdef __cplusplus
}
#endif
#endif /* CCNET_H */
