/* Learned warm start for SPFOM: a small perceptron that predicts the bid
 * prices y (the duals of the resource constraints) from per-resource features
 * of an instance, used as the starting point of spfom_solve.
 *
 * The paper has no counterpart: its conclusion (Section 7) names data-driven
 * modules as future work. The method itself stays the judge: the prediction is
 * only a starting point, the KKT residual of the iteration decides convergence
 * exactly as for a cold start, a prediction whose dual objective is no better
 * than that of y = 0 is discarded, and a warm run that has not converged within
 * its iteration budget is abandoned for a cold start.
 *
 * Network (all sizes fixed): x in R^16 -> h1 = relu(W1 x + b1) in R^256 ->
 * h2 = relu(W2 h1 + b2) in R^256 -> o = w3 . h2 + b3; y_i = max(0, o_i) * mean(r).
 * The matrix products run on the tensor cores in BF16 with FP32 accumulation
 * (inputs, weights and the hidden activations are rounded to BF16 where they
 * enter a product; biases, outputs, the loss and the gradients are FP32).
 * Training minimises the mean squared error (1/R) sum_r (o_r - t_r)^2 with Adam
 * on FP32 master weights.
 *
 * Parameters are one packed FP32 vector of SPFOM_MLP_PARAMS values:
 *   W1 [256][16] row-major | b1 [256] | W2 [256][256] row-major | b2 [256] |
 *   w3 [256] | b3 [1]
 * and gradients use the same layout.
 *
 * Conventions as in spfom.h: every call returns a status; device pointers are
 * caller-owned device memory on the network's device; `stream` NULL means the
 * legacy default stream. Calls on one network must not overlap. */
#ifndef SPFOM_MLP_H
#define SPFOM_MLP_H

#include <stdint.h>

#include "spfom.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SPFOM_MLP_FEATURES 16
#define SPFOM_MLP_HIDDEN 256
#define SPFOM_MLP_PARAMS (256 * 16 + 256 + 256 * 256 + 256 + 256 + 1)

typedef struct spfom_mlp spfom_mlp; /* opaque; owns weights, Adam moments, workspaces */

/* New network on `device`, weights drawn from a seeded uniform
 * +-sqrt(6 / (fan_in + fan_out)) (biases zero). */
spfom_status spfom_mlp_create(int32_t device, uint64_t seed, spfom_mlp** out);
void spfom_mlp_destroy(spfom_mlp* net);

/* Testing aid (no counterpart in the paper): the number of polls after which
 * the tensor-core products' bounded copy waits give up (default 4194304). A
 * wait that gives up sets the network's error flag; the call then returns
 * SPFOM_ETIMEOUT and its outputs are invalid. Before giving up, a block still
 * waits, with the default limit, for the copies it issued and for its issued
 * tensor-core operations, then frees its tensor memory, so no copy or
 * operation is left in flight. A limit of 0 makes every such wait give up at
 * once; tests use it to exercise that path. EINVAL: net is NULL. */
spfom_status spfom_mlp_set_wait_limit(spfom_mlp* net, uint32_t polls);

/* Copy all parameters in (host [SPFOM_MLP_PARAMS]; resets Adam's moments) or out. */
spfom_status spfom_mlp_set_params(spfom_mlp* net, const float* params);
spfom_status spfom_mlp_get_params(spfom_mlp* net, float* params);

/* Gradients of the last spfom_mlp_loss_grad / spfom_mlp_train_step (host [SPFOM_MLP_PARAMS]). */
spfom_status spfom_mlp_get_grads(spfom_mlp* net, float* grads);

/* Outputs o (device [rows] FP32) for the features x (device [rows][16] FP32, row-major). */
spfom_status spfom_mlp_forward(spfom_mlp* net, const float* x, int64_t rows, float* out, void* stream);

/* Forward and backward pass of the loss on (x, t) (t: device [rows] FP32 targets):
 * *loss (host, or NULL) gets the mean squared error; the gradients are kept. */
spfom_status spfom_mlp_loss_grad(spfom_mlp* net, const float* x, const float* t, int64_t rows, double* loss,
                                 void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) with the kept gradients. */
spfom_status spfom_mlp_adam(spfom_mlp* net, float lr, void* stream);

/* spfom_mlp_loss_grad followed by spfom_mlp_adam. */
spfom_status spfom_mlp_train_step(spfom_mlp* net, const float* x, const float* t, int64_t rows, float lr,
                                  double* loss, void* stream);

/* Per-resource features of the single instance loaded in ctx (device [m][16]
 * FP32, row-major, caller-owned), computed on the ctx's stream from the
 * expected sales s(0) of the best assortments at y = 0, d = A s(0), and the
 * prices of the products using each resource:
 *   0 c_i / mean(c)           1 d_i / mean(c)           2 min(c_i / d_i, 4)
 *   3 log(d_i / c_i) in [-6, 6]
 *   4 consumption-weighted mean r_j / mean(r)   5 max r_j / mean(r)
 *   6 consumption-weighted std r_j / mean(r)
 *   7 consumption-weighted mean of r_j / (resources of j) / mean(r)
 *   8 products using i / (nnz(A) / m)           9 sum(c) / sum(d)
 *  10 consumption-weighted mean over the products using i of the largest
 *     min(d_k / c_k, 8) among their resources k
 *  11 1                      12 [d_i > c_i]            13..15 0
 * (weights a_ij s_j(0); empty sums give 0). ESTATE without an instance,
 * ENOTSUP for a batch. */
spfom_status spfom_features(spfom_ctx* ctx, float* features);

/* Solve from the network's prediction: features, forward pass, y0 = max(0, o) mean(r);
 * if Dual(y0) >= Dual(0) the prediction is discarded (cold start, *mode_out = 0);
 * otherwise spfom_solve from y0 with at most warm_iters iterations (<= 0: the
 * ctx's max_iters) -- converged: *mode_out = 1; else a cold spfom_solve from
 * y = 0 with the ctx's max_iters (*mode_out = 2). out->seconds covers the whole
 * call, prediction included. */
spfom_status spfom_solve_warm(spfom_ctx* ctx, spfom_mlp* net, int64_t warm_iters, spfom_stats* out,
                              int32_t* mode_out);

#ifdef __cplusplus
}
#endif

#endif /* SPFOM_MLP_H */
