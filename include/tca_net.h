/*
 * tca_net.h - learned initial guess for the separable tensor-operator solve.
 *
 * The paper solves its tensor equations by plain CG (Sec. 4.1, Fig. 2) and
 * has no learned component; this part of the library adds one around that
 * method.  A small 3D convolutional network, trained on (right-hand side,
 * solution) pairs that the CG solver itself produces, maps A^T b to an
 * initial guess x0; CG then runs from x0 and still decides when the error is
 * small enough (it stops on the same true relative residual as tca_solve).
 *
 * Network (4 layers, 3x3x3 kernels, 32 channels, ReLU):
 *   h1 = relu(conv(u, W1) + b1)    1 -> 32
 *   h2 = relu(conv(h1, W2) + b2)   32 -> 32
 *   h3 = relu(conv(h2, W3) + b3)   32 -> 32
 *   y  = conv(h3, W4) + b4         32 -> 1
 * conv is the 'same' 3x3x3 cross-correlation with zero padding over modes
 * 1..3 of a (D, H, W, B) C-order tensor; mode 4 (B) is a batch index.  The
 * weights and the inter-layer activations are stored in bfloat16 and every
 * sum accumulates in FP32; the master parameters and the Adam moments are
 * FP32.
 *
 * Parameters are exchanged as one packed FP32 host array of
 * tca_net_param_count() values: for each layer W[c_out][c_in][3][3][3]
 * (C order; the last three indices are the offsets -1, 0, +1 in modes 1, 2,
 * 3), then b[c_out].
 *
 * All tensor arguments are FP32 device pointers (TCA_ERR_UNSUPPORTED for
 * host pointers).  Calls are asynchronous on the stream unless noted.  A
 * network object may be used by one stream at a time.
 */
#ifndef TCA_NET_H
#define TCA_NET_H

#include "tca.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tca_net_s* tca_net_t;

/* Number of packed FP32 parameters (57,121). */
TCA_API int64_t tca_net_param_count(void);

/* Create a network with the given packed parameters (host); the Adam state
 * starts at zero.  Synchronises the stream. */
TCA_API tca_status tca_net_create(tca_net_t* out, const float* params, cudaStream_t stream);

/* Replace the parameters (host, packed) and reset the Adam state and the
 * accumulated gradient.  Synchronises the stream. */
TCA_API tca_status tca_net_set_params(tca_net_t net, const float* params, cudaStream_t stream);

/* Copy the master parameters / the accumulated gradient to host memory
 * (packed order).  Synchronises the stream. */
TCA_API tca_status tca_net_get_params(tca_net_t net, float* params, cudaStream_t stream);
TCA_API tca_status tca_net_get_grads(tca_net_t net, float* grads, cudaStream_t stream);

/* y = Net(u); dims = (D, H, W, B), each in 1..65536. */
TCA_API tca_status tca_net_forward(tca_net_t net, const int64_t* dims, const float* u, float* y,
                                   cudaStream_t stream);

/* Forward and backward pass for one pair (u, t) of shape dims: adds
 * L = mean((Net(u) - t)^2) to the loss accumulator and dL/dparams to the
 * gradient accumulator (backpropagation; the gradients with respect to the
 * stored activations are kept in bfloat16 like the activations). */
TCA_API tca_status tca_net_accumulate(tca_net_t net, const int64_t* dims, const float* u, const float* t,
                                      cudaStream_t stream);

/* Read and reset the loss accumulator.  Synchronises the stream. */
TCA_API tca_status tca_net_take_loss(tca_net_t net, double* loss, cudaStream_t stream);

/* One Adam step (Kingma and Ba, 2015; bias-corrected) with gradient
 * grad_scale * (accumulated gradient), then reset the accumulator.
 * lr >= 0, beta1 and beta2 in [0, 1), eps > 0. */
TCA_API tca_status tca_net_adam(tca_net_t net, float lr, float beta1, float beta2, float eps, float grad_scale,
                                cudaStream_t stream);

/* Solve (A^T A + lambda R) x = A^T b like tca_solve, starting from
 * x0 = s Net(A^T b / s) with s the RMS of A^T b (FP32).  With net_every > 0
 * the network is also applied as a preconditioner step: after every
 * net_every CG iterations that did not converge, x += s' Net(r / s') with r
 * the true residual A^T b - K x and s' its RMS, and CG restarts from x.  CG
 * still decides when the error is small enough: the solve stops on the same true relative
 * residual as tca_solve.  info->iters counts all CG iterations,
 * info->refinements the preconditioner steps.  The plan must be FP32 or an
 * _IR precision, of order 3 (B = 1) or 4.  b and x: device pointers.
 * opts->x0_given is ignored.  Synchronises the stream. */
TCA_API tca_status tca_solve_net(tca_plan_t plan, tca_net_t net, const void* b, void* x, const tca_solve_opts* opts,
                                 int net_every, tca_solve_info* info, cudaStream_t stream);

/* Run the 32 -> 32 channel layers (forward and input gradients) on the
 * tensor cores (enable != 0, the default: tcgen05 implicit GEMM, BF16
 * operands, FP32 accumulation in tensor memory) or on the CUDA cores (FP32
 * FMA).  Both compute the same sums; the tensor-core path applies when the
 * batch extent B is at most 24 and falls back to the CUDA cores otherwise. */
TCA_API tca_status tca_net_use_tensor_cores(tca_net_t net, int enable);

/* Free the network (NULL is ignored). */
TCA_API void tca_net_destroy(tca_net_t net);

#ifdef __cplusplus
}
#endif

#endif /* TCA_NET_H */
