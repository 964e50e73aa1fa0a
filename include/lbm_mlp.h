/* C ABI of the jet-trajectory surrogate: a multilayer perceptron from the
 * dimensionless groups of a liquid jet to its leading-edge trajectory and its
 * breakup regime.  The paper measures both (Sec. IV.B: z_LE/D against
 * t* = t u_j0 / D; Sec. IV.C: the regime map on the (Re, Oh) plane with the
 * boundaries Oh = 2.8/Re and Oh = 22/Re) from full simulations; the surrogate
 * is trained on the trajectories of batched simulations (lbm_batch_*) and
 * answers many queries at once.  The paper has no surrogate: this interface
 * serves callers that sweep the regime map.
 *
 * Network: x (n_in) -> depth hidden layers of `width` units with SiLU,
 * z / (1 + exp(-z)) -> a linear output of n_pos + n_cls values
 * (positions, then regime logits).  Loss: w_pos * mean over batch and
 * positions of the squared error + w_cls * mean softmax cross-entropy of the
 * logits.  Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 *
 * Numerics: FP32 master parameters and Adam moments; the matrix products take
 * bfloat16 operands (weights and layer inputs rounded to bfloat16) on the
 * tensor cores and accumulate in FP32; pre-activations, the loss and all
 * reductions are FP32 and deterministic (fixed summation order).
 *
 * Parameter order (flat FP32): for each layer l = 1 .. depth+1, W_l row-major
 * (out x in), then b_l.  All functions return LBM_OK or an error code
 * (lbm.h); arrays may be host or device memory (detected), row-major, batch
 * first.  Work goes on the stream given at creation; calls synchronise before
 * returning host results. */
#ifndef LBM_MLP_H
#define LBM_MLP_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_mlp lbm_mlp;

/* Create a network (parameters uniform in +-1/sqrt(fan_in), from `seed`) for
 * batches of up to max_batch rows.  n_in, width >= 1, depth 1..8,
 * n_pos + n_cls >= 1, n_cls 0..64, width <= 4096.  LBM_ENOMEM if device
 * memory runs out. */
LBM_EXPORT lbm_status lbm_mlp_create(int n_in, int width, int depth, int n_pos, int n_cls, int max_batch,
                                     unsigned long long seed, void* cuda_stream, lbm_mlp** out);
/* Number of FP32 parameters (the length of the flat arrays below). */
LBM_EXPORT size_t lbm_mlp_param_count(const lbm_mlp* m);
/* Replace / read all parameters (flat FP32 in the order above).  Setting
 * resets the Adam state. */
LBM_EXPORT lbm_status lbm_mlp_set_params(lbm_mlp* m, const float* params);
LBM_EXPORT lbm_status lbm_mlp_get_params(lbm_mlp* m, float* params);
/* y (batch x (n_pos + n_cls), FP32) = network(x (batch x n_in, FP32)),
 * 1 <= batch <= max_batch. */
LBM_EXPORT lbm_status lbm_mlp_forward(lbm_mlp* m, const float* x, int batch, float* y);
/* Loss and its gradient with respect to every parameter (flat FP32) for one
 * batch: target (batch x n_pos FP32), label (batch int32 in 0..n_cls-1;
 * ignored when n_cls = 0).  loss and grad may be NULL. */
LBM_EXPORT lbm_status lbm_mlp_loss_grad(lbm_mlp* m, const float* x, const float* target, const int* label,
                                        int batch, float w_pos, float w_cls, float* loss, float* grad);
/* One Adam step of learning rate lr on one batch; *loss (may be NULL) is the
 * loss before the step. */
LBM_EXPORT lbm_status lbm_mlp_train_step(lbm_mlp* m, const float* x, const float* target, const int* label,
                                         int batch, float w_pos, float w_cls, float lr, float* loss);
/* Release the network.  NULL is a no-op. */
LBM_EXPORT void lbm_mlp_free(lbm_mlp* m);

#ifdef __cplusplus
}
#endif

#endif
