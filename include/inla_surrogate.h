/*
 * inla_surrogate.h -- C ABI of the learned surrogate of log pi~(theta|y) (the paper has no
 * counterpart: this is the build's learned part).  A multilayer perceptron
 *     f(x) = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3,   x in R^D (D <= 8), hidden width 128,
 * trained on the GPU by full-batch Adam on the mean squared error against exact
 * evaluations (inputs and targets standardised by the caller).  FP32 weights and arithmetic.
 * Parameters are packed as W1 (128 x D, row-major), b1 (128), W2 (128 x 128), b2 (128),
 * w3 (128), b3 (1).
 *
 * Conventions: every function returns INLA_OK (0) or a negative INLA_E_* code of inla.h;
 * every array argument is a caller-owned HOST array, read or written only during the call.
 * A network lives on the device that is current at inla_mlp_create and must be used with
 * that device current, by one host thread at a time.
 */
#ifndef INLA_SURROGATE_H
#define INLA_SURROGATE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define INLA_MLP_HIDDEN 128
#define INLA_MLP_MAX_DIN 8

typedef struct inla_mlp inla_mlp;   /* opaque; owns its device buffers */

/* Number of packed parameters of a network with `din` inputs. */
int64_t inla_mlp_num_params(int32_t din);

/* Allocate a network for `din` inputs (1..8) and batches of up to `max_samples` samples.
 * Parameters start at zero (set them with inla_mlp_set_params).  INLA_E_BADARG, INLA_E_NOMEM. */
int inla_mlp_create(int32_t din, int32_t max_samples, inla_mlp **out);
int inla_mlp_destroy(inla_mlp *net);

/* Copy all parameters in (resetting the Adam moments and step count) or out. */
int inla_mlp_set_params(inla_mlp *net, const float *params);
int inla_mlp_get_params(const inla_mlp *net, float *params);

/* `epochs` full-batch Adam steps (learning rate lr, beta1 0.9, beta2 0.999, eps 1e-8) on the
 * N samples X (N x din, row-major) with targets y (N).  loss_out (epochs floats, may be NULL)
 * receives the loss before each step.  The epoch (forward, backward, update) is one CUDA
 * graph, replayed `epochs` times.  N <= max_samples. */
int inla_mlp_train(inla_mlp *net, const float *X, const float *y, int32_t N, int32_t epochs, float lr,
                   float *loss_out);

/* Mean squared error at the current parameters and its gradient (inla_mlp_num_params
 * floats), without an update. */
int inla_mlp_loss_grad(inla_mlp *net, const float *X, const float *y, int32_t N, float *loss, float *grad);

/* Network outputs f (N) and, when dfdx is not NULL, the input gradients (N x din). */
int inla_mlp_predict(inla_mlp *net, const float *X, int32_t N, float *f, float *dfdx);

#ifdef __cplusplus
}
#endif
#endif /* INLA_SURROGATE_H */
