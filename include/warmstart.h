/*
 * warmstart.h -- C ABI of the learned initial guess for the MAC Stokes MG-SQMR solver (sm_103a).
 *
 * The paper's SQMR (Alg. 4) starts from a given x0 (its experiments use x0 = 0).  This module
 * predicts x0 from the right-hand side b with a small 3D convolutional network trained on
 * solutions the solver itself produced; SQMR with the unchanged symmetric V-cycle preconditioner
 * then runs from that guess (warmstart_solve), so the tolerance reached never depends on the
 * network.  The paper has no such network: the map below is this library's definition.
 *
 * NETWORK (n^3 cube, n a multiple of 8; four levels n, n/2, n/4, n/8; 16 channels; 3x3x3
 * convolutions with zero padding and no bias; leaky ReLU with slope 0.1):
 *   X0 = cells(b) / rms(b)            4 channels per cell: the mean of the cell's two faces for each
 *                                     velocity component, the cell's pressure entry; rms(b) =
 *                                     sqrt(mean of b^2 over the packed vector)
 *   a0 = act(conv(X0, W0)), s0 = act(conv(a0, W1))
 *   a1 = act(conv(pool(s0), W2)), s1 = act(conv(a1, W3))          pool: mean of 2x2x2 cells
 *   a2 = act(conv(pool(s1), W4)), s2 = act(conv(a2, W5))
 *   a3 = act(conv(pool(s2), W6)), b3 = act(conv(a3, W7))
 *   c2 = act(conv(up(b3) + s2, W8)), c1 = act(conv(up(c2) + s1, W9))   up: nearest-neighbour x2
 *   c0 = act(conv(up(c1) + s0, W10)), P = c0 W11 (1x1x1, 16 -> 4 channels)
 *   x0 = scale * rms(b) * faces(P)    interior face = mean of its two cells, wall face 0, pressure P
 * Loss for training (x* = the solver's solution for b): ||x0 - x*||^2 / ||x*||^2, or
 * ||L (x0 - x*)||^2 / ||b||^2 with the problem's operator L (warmstart_loss_grad).
 * WEIGHTS: one flat FP32 vector of warmstart_num_weights() entries: W0 [27][4][16], W1..W10
 * [27][16][16], W11 [16][4]; tap t = 9 (dz+1) + 3 (dy+1) + (dx+1); last index fastest.
 * STORAGE: activations are kept as FP32 or BF16 (WARMSTART_STORE_*); every convolution accumulates
 * in FP32; gradients, weights and Adam moments are FP32.
 * ENGINE: with BF16 storage the 3x3x3 convolutions, their data gradients and weight gradients take
 * BF16 operands on the tensor cores (weights and FP32 gradients rounded to BF16 where they enter a
 * product); with FP32 storage, or warmstart_set_engine(ws, 0), they run in FP32 on the CUDA cores.
 *
 * POINTERS: b, x0, xstar, x are packed FP64 device vectors (layout of stokesmg.h); weight and
 * gradient arrays may be host or device memory.  The handle owns its activation, gradient,
 * moment and scratch buffers.  ERRORS: the STOKES_* codes of stokesmg.h.  A handle is not
 * thread-safe.
 */
#ifndef WARMSTART_H
#define WARMSTART_H

#include "stokesmg.h"

#ifdef __cplusplus
extern "C" {
#endif

#define WARMSTART_STORE_FP32 0
#define WARMSTART_STORE_BF16 1

typedef struct warmstart_s *warmstart_t;

/* flat weight count of the network (70,912) */
long long warmstart_num_weights(void);

/* network for n^3 cells (8 <= n <= 1016, n % 8 == 0) with activation storage `storage` and output
 * scale `scale` (> 0); weights start at 0 (set them before use) */
int warmstart_create(int n, int storage, double scale, warmstart_t *out);
int warmstart_destroy(warmstart_t ws);
int warmstart_set_scale(warmstart_t ws, double scale);
/* tensor_cores = 1 (default) or 0: where BF16-storage convolutions run (see ENGINE) */
int warmstart_set_engine(warmstart_t ws, int tensor_cores);

/* copy num_weights FP32 weights in (resets the Adam moments and step count) / out; synchronous */
int warmstart_set_weights(warmstart_t ws, const float *w);
int warmstart_get_weights(warmstart_t ws, float *w);

/* x0 = network(b) (packed, 0 on the wall-normal faces) */
int warmstart_predict(warmstart_t ws, const double *b, double *x0, void *stream);

/* forward + loss + backward for right-hand side b and the method's solution xstar of it (device
 * vectors).  h == NULL: loss ||x0 - x*||^2 / ||x*||^2; h = the n^3 Stokes handle of the problem:
 * loss ||L (x0 - x*)||^2 / ||b||^2 (what SQMR's stopping test measures; two stokes_apply calls).
 * The gradient goes into the handle's gradient buffer and, if grad != NULL, is copied to grad (host
 * or device, num_weights floats; synchronises).  If loss != NULL the stream is synchronised and
 * *loss receives the loss. */
int warmstart_loss_grad(warmstart_t ws, stokes_t h, const double *b, const double *xstar, double *loss, float *grad,
                        void *stream);

/* one Adam update (Kingma & Ba, Algorithm 1) of the weights from the handle's gradient buffer */
int warmstart_adam_step(warmstart_t ws, double lr, double beta1, double beta2, double eps, void *stream);

/* Tensor-core kernels report a bounded wait that ran out as STOKES_ERR_TIMEOUT from the next call that
 * synchronises (warmstart_loss_grad with loss or grad, warmstart_solve). */

/* SQMR solve of stokes handle h from the network's guess: x <- network(b); the guess is kept only
 * if it lowers both the residual (||b - L x|| < ||b||) and SQMR's first quantity tau_0 =
 * ||M (b - L x)|| (Alg. 4, M = the V-cycle) below its value for x0 = 0, ||M b||; otherwise x <- 0.
 * Then sqmr_solve(h, b, x, tol, max_iter, info).  Costs one network evaluation, one operator apply
 * and two V-cycles before the solve.
 * *used_guess (may be NULL) tells which start was taken.  h must be an n^3 problem on the same
 * device. */
int warmstart_solve(warmstart_t ws, stokes_t h, const double *b, double *x, double tol, int max_iter,
                    sqmr_info_t *info, int *used_guess, void *stream);

/* ---- checks of single network operations (device pointers; synchronous) ----
 * op 0: out (BF16 [n^3][16]) = act(conv(x (BF16 [n^3][ci]), w [27][ci][16]))
 * op 1: out (FP32 [n^3][16]) = data gradient of a 16 -> 16 layer w [27][16][16] for the output
 *       gradient x (FP32 [n^3][16]): out[v] = sum_t x[v - off_t] w[t]^T
 * op 2: out (FP32 [27][ci][16]) = weight gradient sum_v x[v + off_t][ci] g[v][co] (x BF16 [n^3][ci],
 *       g FP32 [n^3][16])
 * ci is 4 or 16 (16 for op 1); engine 0 = CUDA cores (FP32 arithmetic), 1 = tensor cores (BF16
 * operands, FP32 accumulation; STOKES_ERR_UNSUPPORTED where that form does not apply). */
int warmstart_conv_check(int n, int ci, int op, int engine, const void *x, const float *g, const float *w, void *out,
                         void *stream);
/* one tcgen05 tensor-core MMA: d (FP32 [128][16]) = a (BF16 [128][16]) b^T (b BF16 [16][16], [n][k]) */
int warmstart_mma_check(const void *a, const void *b, float *d, void *stream);

#ifdef __cplusplus
}
#endif

#endif
