/*
 * lisa_flow.h -- C ABI of the normalizing-flow proposal used by the ensemble sampler
 * (lisa_sampler.h).  The flow is not part of Katz et al. (2020): it is an independence
 * proposal for the Metropolis-Hastings rule of Eq. (13), whose acceptance
 * min(1, L(y)/L(x) Q(x)/Q(y)) keeps the chain exact whatever the proposal density Q.
 *
 * Flow (over the 11 sampling coordinates of Table I):
 *   u = L^{-1} (x - mu) (mu: mean of the training set, L L^T: its covariance, L lower
 *   triangular, each Cholesky pivot floored at 1e-12 of its diagonal entry); eight
 *   affine coupling layers; layer c keeps the coordinates with
 *   mask m_c = 1 (c mod 4 = 0: even coordinates, 1: odd, 2: coordinates 0..5,
 *   3: coordinates 6..10) and maps the others by v = (u - t) e^{-s}, where
 *   s = 2 tanh(o_s / 2), t = o_t and (o_s, o_t) = W3 relu(W2 relu(W1 (m u) + b1) + b2) + b3
 *   (11 -> 128 -> 128 -> 22).  z = layers(u) is standard normal under the flow:
 *   log q(x) = -|z|^2/2 - (11/2) log 2 pi - sum_c sum_d s_cd - sum_d log L_dd.
 *
 * Arithmetic: the three GEMMs of every layer (and, in training, the six of its
 * backward pass) run on the tensor cores with bfloat16 operands and FP32 accumulation
 * (mma.sync m16n8k16); the coupling update, log-determinant and loss are FP32, the
 * whitening and log q totals FP64.  Master weights and Adam moments are FP32.
 *
 * Weights, host layout [8][20886] floats, per coupling:
 *   W1 [128][11], b1 [128], W2 [128][128], b2 [128], W3 [22][128], b3 [22]
 * with rows of W3 ordered (o_s for coordinates 0..10, o_t for coordinates 0..10).
 *
 * Every function returns a lisa_status; messages via lisa_flow_last_error.  Device
 * pointers are FP64 rows of 11 values.  Functions taking a stream enqueue on it (NULL =
 * the default stream) and return without waiting unless stated.
 */
#ifndef LISA_FLOW_H
#define LISA_FLOW_H

#include <stdint.h>

#include "lisa_like.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LISA_FLOW_DIM 11
#define LISA_FLOW_COUPLINGS 8
#define LISA_FLOW_HIDDEN 128
#define LISA_FLOW_PARAMS_PER_COUPLING 20886

typedef struct lisa_flow lisa_flow_t;

/* New flow on the current device: hidden layers uniform in +-sqrt(6 / fan_in) from a
 * Philox stream keyed by seed, zero biases, zero output layer (the identity map), and
 * mu = 0, L = I. */
lisa_status lisa_flow_create(uint64_t seed, lisa_flow_t **out);
void lisa_flow_destroy(lisa_flow_t *f);
const char *lisa_flow_last_error(const lisa_flow_t *f);

/* Master weights to/from host memory ([8][20886] floats, layout above). Synchronous. */
lisa_status lisa_flow_set_weights(lisa_flow_t *f, const float *w);
lisa_status lisa_flow_get_weights(lisa_flow_t *f, float *w);

/* Whitening mu [11] and L [11][11] row-major, lower triangular with a positive diagonal
 * (entries above the diagonal are ignored and read back as 0).  Synchronous. */
lisa_status lisa_flow_set_whitening(lisa_flow_t *f, const double *mu, const double *L);
lisa_status lisa_flow_get_whitening(lisa_flow_t *f, double *mu, double *L);

/* x [n][11] -> z [n][11] (may be NULL) and log q(x) [n]. */
lisa_status lisa_flow_normalize(lisa_flow_t *f, const double *d_x, int n, double *d_z,
                                double *d_logq, void *stream);

/* z [n][11] -> x [n][11] and log q(x) [n]. */
lisa_status lisa_flow_generate(lisa_flow_t *f, const double *d_z, int n, double *d_x,
                               double *d_logq, void *stream);

/* Mean of -log q_u(u) + const (the training loss) over the batch d_x [n][11],
 * whitened with the flow's current mu, L, and its gradient with respect to
 * every weight (host grad [8][20886], may be NULL).  n must be a multiple of 64.
 * Synchronous. */
lisa_status lisa_flow_gradients(lisa_flow_t *f, const double *d_x, int n, float *grad,
                                double *loss, void *stream);

/* Train on d_data [n][11]: set mu, L from the data, reset the Adam moments, then
 * `iters` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on
 * minibatches of `batch` rows (a multiple of 64) drawn with Philox counters
 * (round, 5, iteration, row / 4) keyed by seed.  loss (host [iters], may be NULL)
 * receives each step's minibatch loss.  Synchronous. */
lisa_status lisa_flow_train(lisa_flow_t *f, const double *d_data, int64_t n, int iters,
                            int batch, double lr, uint64_t seed, uint32_t round, double *loss,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif
