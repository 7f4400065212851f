/*
 * perm_mlp.h -- the learned cost model that perm_auto uses in place of the paper's
 * compile-time tuned hyperplanes (Algorithm "Optimized Algorithm Selection"): a
 * three-layer FP32 perceptron
 *     h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3
 * that predicts log2(seconds) of each candidate algorithm from features of the
 * matrix (perm_auto_features), trained on the GPU by the kernels below on timings
 * that this library measures itself.
 *
 * Weights are one flat float array: W1 [in x hidden] (row-major), b1 [hidden],
 * W2 [hidden x hidden], b2 [hidden], W3 [hidden x out], b3 [out];
 * perm_mlp_size gives its length.  Limits: 1 <= in <= 64, 1 <= hidden <= 256,
 * 1 <= out <= 64.  All arrays of the training and gradient calls are device memory
 * (float32, row-major, `rows` rows); loss_history may be device or host memory.
 */
#ifndef PERM_MLP_H_
#define PERM_MLP_H_

#include <stdint.h>

#include "perm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Candidates perm_auto chooses between (output index of the cost model): an algorithm
 * with a kernel configuration (arithmetic, how chunk starts are formed, chunk length). */
typedef enum {
  PERM_CAND_COMBINATORIC = 0, /* perm_combinatoric */
  PERM_CAND_RYSER = 1,        /* perm_ryser, default arithmetic (real: integer pipes from n = 10 or the
                                 by-size walk; complex FP64; integers exact) */
  PERM_CAND_GLYNN = 2,        /* perm_glynn, FP64 (real), default (complex), exact (integers) */
  PERM_CAND_GLYNN_FIXED = 3,  /* perm_glynn, PERM_ARITH_MIXED: integer pipes with a share of each product
                                 on the FP64 unit (real input) */
  PERM_CAND_RYSER_FP64 = 4,   /* perm_ryser, PERM_ARITH_FP64 (real input) */
  PERM_CAND_GLYNN_DMMA = 5,   /* perm_glynn, PERM_ARITH_FP64 with chunk starts from the FP64 tensor-core
                                 contraction (real input, n <= 48) */
  PERM_CAND_GLYNN_INT = 6,    /* perm_glynn, PERM_ARITH_FIXED: integer pipes only (real input) */
  PERM_CAND_GLYNN_SHORT = 7,  /* perm_glynn, PERM_ARITH_MIXED with chunks of 2^6 terms (real), or
                                 PERM_ARITH_FP64 (complex) */
  PERM_NCAND = 8,
  PERM_CAND_CAUCHY = 8        /* not a cost-model output: a real square matrix of order >= 24 whose
                                 entries are 1/(x_i - y_j) within 2^-48 relative, all of one sign,
                                 is evaluated by Borchardt's theorem on the fitted points (see
                                 perm_cauchy); the error bound then adds n 2^-48 (1 + n 2^-48) |per| */
} perm_candidate;

#define PERM_NFEATURES 12

/* Features of an m x n matrix (after the transpose rule) with a fraction `density`
 * of nonzero entries: writes PERM_NFEATURES floats to `out` (host memory). */
int perm_auto_features(int64_t m, int64_t n, double density, int dtype, float* out);

/* Number of floats in the flat weight array. */
int perm_mlp_size(int32_t in_dim, int32_t hidden, int32_t out_dim, int64_t* count);

/* y = MLP(X) for `rows` feature rows. */
int perm_mlp_forward(const float* weights, int32_t in_dim, int32_t hidden, int32_t out_dim, const float* X,
                     int64_t rows, float* Y, void* stream);

/* Gradient of the masked mean squared error
 *     L = sum_{r,k} mask[r,k] (y[r,k] - T[r,k])^2 / sum mask
 * with respect to the flat weights (written to grad, same layout), and L to *loss
 * (device pointer, may be null). */
int perm_mlp_grad(const float* weights, int32_t in_dim, int32_t hidden, int32_t out_dim, const float* X,
                  const float* T, const float* mask, int64_t rows, float* grad, float* loss, void* stream);

/* Initialise the weights from `seed` (uniform He-style, counter-based) and train with
 * Adam (beta1 0.9, beta2 0.999) on mini-batches of `batch` consecutive rows for
 * `epochs` passes; the loss of each epoch's last mini-batch goes to loss_history[ep]
 * (if not null). */
int perm_mlp_train(const float* X, const float* T, const float* mask, int64_t rows, int32_t in_dim, int32_t hidden,
                   int32_t out_dim, int32_t epochs, int32_t batch, float lr, uint64_t seed, float* weights,
                   float* loss_history, void* stream);

/* Install a trained model (host weights, copied) in the handle for perm_auto;
 * weights = NULL removes it (perm_auto then uses its built-in rule). */
int perm_set_cost_model(perm_handle h, const float* weights, int32_t in_dim, int32_t hidden, int32_t out_dim);

/* The choice perm_auto would make for this matrix (no permanent is computed): *candidate
 * gets a perm_candidate, predicted (if not null) PERM_NCAND predicted log2 seconds
 * (+inf for candidates that are not available or exceed the work cap; all +inf for
 * PERM_CAND_CAUCHY). */
int perm_auto_choice(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, const perm_opts* opts,
                     int* candidate, float* predicted);

#ifdef __cplusplus
}
#endif

#endif /* PERM_MLP_H_ */
