/*
 * lisa_sampler.h -- C ABI of the parallel-tempered affine-invariant ensemble sampler
 * that consumes the batched likelihood of lisa_like.h (Katz et al. 2020, Sec. III).
 *
 * One step of the sampler, every part of it a CUDA kernel on the likelihood handle's
 * stream (one CUDA graph per step when graphs are on):
 *   1. stretch proposals for the first half of every temperature's walkers
 *      (Sec. III.A, Eqs. (14)-(15)): partner from the other half, y = x_j + z (x_k - x_j),
 *      z drawn from g(z) ~ 1/sqrt(z) on [1/a, a];
 *   2. the batched ln L of all T * W/2 proposals (lisa_like.h), or a Gaussian test target;
 *   3. acceptance with probability min(1, z^(D-1) [L(y)/L(x)]^beta pi(y)/pi(x)) (Eq. (16)
 *      with the tempered likelihood L^beta of Sec. III.B, D = 11);
 *   4. steps 1-3 for the second half;
 *   5. temperature swaps between walker w of adjacent temperatures with probability
 *      min(1, [L_hot/L_cold]^(beta_cold - beta_hot)) (Eq. (17)), from the hottest pair down;
 *   6. optionally the adaptive ladder of Vousden, Farr & Mandel (2016);
 *   7. the coldest temperature's positions and ln L appended to the caller's chain.
 *
 * Sampling coordinates (Table I), in this order:
 *   x = (ln M_T, q, a1, a2, ln D_L, phi_ref, cos iota, lambda, sin beta, psi, ln t_ref)
 * with a uniform prior inside [lower, upper] (Table I bounds by default).  With
 * lisa_frame set, lambda, beta, psi and t_ref are LISA-frame values that are converted
 * to the SSB frame before the likelihood (Sec. II).  The LISA frame is the frame in which
 * the rigid constellation of the response model is at rest, taken at the signal's arrival
 * time at the constellation centre, t_L = t_SSB + k . p0(t_SSB).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011) keyed by the seed,
 * counter (step, phase, temperature, walker), phase 0/1 for the two halves and 2 for the
 * swaps; uniforms (u + 0.5) 2^-32.  A run is reproducible from (seed, step, state).
 *
 * Arrays: x [T][W][11] row-major FP64, ln L [T][W], betas [T] (beta_0 = 1 is the target
 * distribution), counters [T][2] = (accepted, proposed).  Temperature 0 is the coldest.
 *
 * Errors: every function returns a lisa_status; the message is read with
 * lisa_sampler_last_error.  A likelihood call that gave up on a device wait (the
 * likelihood's LISA_ERR_TIMEOUT) poisons the run: the sampler accepts nothing more and
 * lisa_sampler_run returns LISA_ERR_TIMEOUT.  Not thread-safe per handle.
 */
#ifndef LISA_SAMPLER_H
#define LISA_SAMPLER_H

#include <stdint.h>

#include "lisa_flow.h"
#include "lisa_like.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LISA_SAMPLER_NDIM 11
#define LISA_SAMPLER_MAX_TEMPS 64

typedef struct lisa_sampler lisa_sampler_t;

typedef enum {
    LISA_TARGET_LIKELIHOOD = 0, /* the batched LISA ln L of the lisa_like handle */
    LISA_TARGET_GAUSSIAN = 1    /* N(gauss_mean, diag(gauss_sigma^2)), for checking the sampler */
} lisa_target;

typedef struct {
    int n_temps;          /* T, 1..LISA_SAMPLER_MAX_TEMPS */
    int n_walkers;        /* W per temperature, even, >= 4 */
    double a;             /* stretch scale of Eq. (15); 1.15 as in Sec. III.B */
    double ladder_ratio;  /* T_{t+1} / T_t of the default ladder: 2.04807 for D = 11 */
    int t_max_inf;        /* 1: the hottest temperature is infinite (beta = 0), Sec. III.B */
    int adaptive;         /* 1: Vousden et al. ladder adaptation after every step */
    double adapt_lag;     /* t0 of kappa(s) = t0 / (nu (s + t0)) */
    double adapt_time;    /* nu */
    uint64_t seed;        /* Philox key */
    double lower[LISA_SAMPLER_NDIM], upper[LISA_SAMPLER_NDIM]; /* prior box (Table I) */
    int lisa_frame;       /* 1: sky position, polarisation, t_ref in the LISA frame */
    int target;           /* lisa_target */
    double gauss_mean[LISA_SAMPLER_NDIM], gauss_sigma[LISA_SAMPLER_NDIM];
    int use_graphs;       /* 1: each step replays one captured CUDA graph */
    double timeout_s;     /* host wait bound per step; <= 0: the likelihood's (else 60 s) */
} lisa_sampler_config;

/* Defaults: T = 8, W = 256, a = 1.15, ratio 2.04807, t_max_inf = 1, adaptive = 1,
 * t0 = 10000, nu = 100, seed 1, Table I bounds, lisa_frame = 1, likelihood target,
 * graphs on, timeout_s = 0. */
void lisa_sampler_default_config(lisa_sampler_config *cfg);

/* Create a sampler.  `like` must have data set (lisa_like_set_data) and
 * max_batch >= T * W / 2; it may be NULL for the Gaussian target.  The sampler borrows
 * `like` (and its stream): destroy the sampler first.  The ladder starts as
 * beta_t = ratio^-t with beta_{T-1} = 0 when t_max_inf.  Errors: LISA_ERR_ARG (config),
 * LISA_ERR_STATE (no data), LISA_ERR_CUDA / LISA_ERR_OOM. */
lisa_status lisa_sampler_create(lisa_like_t *like, const lisa_sampler_config *cfg,
                                lisa_sampler_t **out);

/* Replace the ladder: betas [T] host, 1 >= beta_0 > beta_1 > ... >= 0. */
lisa_status lisa_sampler_set_ladder(lisa_sampler_t *s, const double *betas);

/* Set the walkers (host x [T][W][11]) and the step counter of the next step, and
 * evaluate their ln L (points outside the prior get -inf).  Synchronous. */
lisa_status lisa_sampler_set_state(lisa_sampler_t *s, const double *x, uint32_t step);

/* Run n_steps >= 1 steps.  d_chain (device [n_steps][W][11]) and d_lnl (device
 * [n_steps][W]) receive the coldest temperature after each step; either may be NULL.
 * Synchronous: returns when the steps are done (LISA_ERR_TIMEOUT after
 * n_steps x timeout_s, or when a likelihood call gave up). */
lisa_status lisa_sampler_run(lisa_sampler_t *s, int n_steps, double *d_chain, double *d_lnl);

/* Current state to host buffers (any may be NULL): x [T][W][11], lnl [T][W],
 * betas [T], step = the counter of the next step. */
lisa_status lisa_sampler_get_state(lisa_sampler_t *s, double *x, double *lnl, double *betas,
                                   uint32_t *step);

/* Accumulated stretch and swap counts since set_state: acc [T][2], swaps [T][2] as
 * (accepted, proposed); swaps of pair (t, t+1) are stored at t. */
lisa_status lisa_sampler_get_counts(lisa_sampler_t *s, int64_t *acc, int64_t *swaps);

/* Kernels launched per step (proposal, likelihood, acceptance and swap kernels). */
int lisa_sampler_step_launches(const lisa_sampler_t *s);

void lisa_sampler_destroy(lisa_sampler_t *s);
const char *lisa_sampler_last_error(const lisa_sampler_t *s);

/* Flow proposal (lisa_flow.h) for the coldest temperature.  Once active, every step
 * starts with one independence Metropolis-Hastings move of each coldest walker
 * (Eq. (13)): y = flow(z), z from Philox counters (step, 3, blk, w), blk = 0..2, by
 * Box-Muller in pairs (the first 11 of 12 normals); accepted with probability
 * min(1, [L(y)/L(x)]^beta_0 pi(y)/pi(x) q(x)/q(y)), the uniform from counter
 * (step, 4, 0, w); the batched ln L of the W proposals runs inside the step's graph.
 * Training: after every train_every steps (counted from set_state) the flow is fitted
 * to the coldest walkers of those steps (lisa_flow_train: train_iters Adam steps on
 * minibatches of `batch` rows, round = number of earlier trainings, key = seed); the
 * proposals start after the first training.  No training after freeze_after steps
 * (0: never stop); train_every = 0: never train, the flow's current weights propose
 * from the first step (set them through lisa_sampler_get_flow).  flow_only = 1 skips the
 * stretch moves and temperature swaps. */
typedef struct {
    int train_every;   /* 500 */
    int train_iters;   /* 400 */
    int batch;         /* 1024, a multiple of 64 */
    double lr;         /* 1e-3 */
    int freeze_after;  /* 0 */
    uint64_t seed;     /* weight initialisation and minibatch draws: 1 */
    int flow_only;     /* 0 */
} lisa_flow_schedule;

void lisa_flow_default_schedule(lisa_flow_schedule *fs);

/* Enable the flow (once per sampler; the likelihood's max_batch must be >= W).
 * Counters and the training schedule restart at the next set_state. */
lisa_status lisa_sampler_enable_flow(lisa_sampler_t *s, const lisa_flow_schedule *fs);

/* The sampler's flow (borrowed; NULL before lisa_sampler_enable_flow). */
lisa_flow_t *lisa_sampler_get_flow(lisa_sampler_t *s);

/* Evaluate the flow moves' proposals with another likelihood handle (borrowed, same
 * device, same data and t0 as the sampler's, max_batch >= W), e.g. an FP64 handle for
 * exact acceptances while the stretch moves use a split-precision one; NULL restores the
 * sampler's own.  Requires lisa_sampler_enable_flow. */
lisa_status lisa_sampler_set_flow_likelihood(lisa_sampler_t *s, lisa_like_t *like2);

/* Screen the flow moves (margin > 0, in ln L units; 0 turns the screen off).  Every flow
 * proposal is first evaluated by the sampler's own likelihood; a proposal whose
 * Metropolis-Hastings log ratio (Eq. (13) with the proposal density) falls below log u by
 * more than beta_0 * margin is rejected there, and every other one is evaluated by the
 * second likelihood (lisa_sampler_set_flow_likelihood), whose ln L decides it and is the
 * one stored on acceptance.  The chain equals the unscreened chain of the second
 * likelihood whenever the two likelihoods differ by less than margin at the rejected
 * proposals (e.g. split precision against FP64: |d lnL| ~1e-4 near the posterior at SNR
 * 1000), while the second likelihood works only on the proposals sent on.  Needs a
 * second likelihood; LISA_ERR_STATE otherwise, LISA_ERR_ARG for a negative or
 * non-finite margin. */
lisa_status lisa_sampler_set_flow_screen(lisa_sampler_t *s, double margin);

/* Flow proposals sent to the second likelihood by the screen since set_state. */
lisa_status lisa_sampler_flow_screen_count(lisa_sampler_t *s, int64_t *sent);

/* acc [2] = (accepted, proposed) flow moves since set_state; trainings so far; the last
 * minibatch loss of the last training (NaN before the first).  Any may be NULL. */
lisa_status lisa_sampler_flow_stats(lisa_sampler_t *s, int64_t *acc, int *trainings,
                                    double *last_loss);

/* Sampling coordinates -> the physical parameter vector of lisa_like.h, on the device:
 * d_x [n][11] -> d_th [n][11], with the LISA-frame conversion when lisa_frame, absolute
 * times t = t_ref + t0.  Points are converted as given (no prior check).  Enqueued on
 * `stream` (NULL = default stream); asynchronous. */
lisa_status lisa_sampler_to_physical(const double *d_x, int n, int lisa_frame, double t0,
                                     double *d_th, void *stream);

/* The inverse on the host: physical parameters th [n][11] (SSB frame, t_ref relative to
 * t0) -> sampling coordinates x [n][11], with lambda, sin beta, psi and ln t_ref in the
 * LISA frame when lisa_frame (t_L = t + k . p0(t), then the constellation frame at t_L).
 * LISA_ERR_ARG when a parameter has no sampling coordinate (M_T, D_L or the reference
 * time not positive). */
lisa_status lisa_sampler_from_physical(const double *th, int n, int lisa_frame, double t0,
                                       double *x);

/* Initial walkers at the 8 LISA-frame sky modes of Sec. III.B: walker w of every
 * temperature sits at mode w % 8, longitude lambda_L + (w % 4) pi/2 (wrapped into the
 * prior range) and sin beta_L with sign flipped for (w / 4) % 2 = 1, plus a Gaussian
 * jitter of standard deviation scale[i] per coordinate, reflected back into the prior
 * box.  Host only; x_out [T][W][11]; seed keys a Philox stream.  W must be a multiple
 * of 8. */
lisa_status lisa_sampler_sky_mode_init(const double *x_center, const double *scale,
                                       const double *lower, const double *upper, int T, int W,
                                       uint64_t seed, double *x_out);

/* Integrated autocorrelation time of Sec. III.C (Eqs. (19)-(22)) of one coordinate on
 * the device: the series is d_chain[(i * W + w) * stride + offset] for step i < n and
 * walker w < W.  The per-walker normalised autocorrelation (1/(N - tau) estimator) is
 * averaged over walkers; tau(M) = 1 + 2 sum_{t<=M} rho(t) at the smallest M with
 * M >= 5 tau(M).  rho (host [n], may be NULL) receives rho(0..M) and zeros beyond.
 * Synchronous on `stream` (NULL = default stream). */
lisa_status lisa_autocorr_time(const double *d_chain, int n, int W, int stride, int offset,
                               double *tau, double *rho, void *stream);

#ifdef __cplusplus
}
#endif
#endif
