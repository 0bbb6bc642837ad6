/*
 * lisa_like.h -- C ABI of liblisalike.so: the batched LISA log-likelihood for
 * massive-black-hole-binary templates (Katz, Marsat, Chua, Babak & Larson 2020),
 * computed on one GB300 GPU.
 *
 * What one call computes (Sec. II and II.A of the paper), for every walker b:
 *   1. the harmonic amplitude A_lm(f) and phase phi_lm(f) of Eq. (5) on K
 *      log-spaced knots spanning the mode's band; t_lm(f) of Eq. (6) and the cut
 *      where t_lm(f) < 0;
 *   2. the TDI A/E/T transfer T(f, t_lm(f)) of Eqs. (7)-(10) at those knots;
 *   3. not-a-knot cubic splines of A, phi and T onto the dense grid f_j = f0 + j df;
 *   4. the sum over modes of T A e^{i(phi - 2 pi f t_coal)} (never stored);
 *   5. <d|h> and <h|h> of Eqs. (3) and (11), and ln L = <d|h> - <h|h>/2 - <d|d>/2
 *      of Eq. (2).
 * The waveform and response coefficients are stand-ins of the paper's functional
 * forms (the paper defers the fits to cited work); see the project design notes.
 *
 * Conventions used by every entry point:
 *   - Parameters are double[B][11] rows in the paper's order (Sec. II):
 *     M_T [M_sun, detector frame], q (<= 1), a1, a2, D_L [Gpc], phi_ref, iota,
 *     lambda, beta, psi (SSB frame, rad), t_ref [s]; t_coal = t_ref + t0.
 *   - Channel arrays are ordered A, E, T; complex values are interleaved (re, im).
 *   - A walker with M_T <= 0, q outside (0, 1], |a_i| > 0.99, D_L <= 0 or any
 *     non-finite entry gets ln L = -inf, <d|h> = <h|h> = 0; the status stays OK.
 *   - A walker whose bands miss the grid has h = 0 and ln L = -<d|d>/2.
 *   - On a non-OK status nothing is written to the outputs and
 *     lisa_like_last_error() describes the failure.
 *   - One handle per host thread; calls on one handle are serialised on its stream.
 * Ownership: the library owns all device memory it allocates, until
 * lisa_like_destroy(); inputs are copied; outputs are caller-allocated.
 */
#ifndef LISA_LIKE_H
#define LISA_LIKE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lisa_like lisa_like_t;

typedef enum {
    LISA_OK = 0,
    LISA_ERR_ARG = 1,     /* invalid argument (NULL, size, non-finite, bad mode ...) */
    LISA_ERR_STATE = 2,   /* call out of order (e.g. loglike before set_data) */
    LISA_ERR_CUDA = 3,    /* a CUDA runtime call failed */
    LISA_ERR_OOM = 4,     /* device or pinned-host allocation failed */
    LISA_ERR_TIMEOUT = 5  /* a bounded wait for the device gave up */
} lisa_status;

enum { LISA_PREC_FP64 = 0, LISA_PREC_SPLIT = 1 };

#define LISA_NPAR 11
#define LISA_MAX_MODES 6
#define LISA_NSERIES 8

typedef struct {
    int n_modes;            /* 1..6 */
    int modes[6][2];        /* (l,m) pairs from (2,2),(3,3),(4,4),(2,1),(3,2),(4,3) */
    int n_knots;            /* K >= 4 knots per mode (not-a-knot needs 4); paper: ~2^10 */
    int precision;          /* LISA_PREC_FP64 or LISA_PREC_SPLIT */
    double t0_s;            /* t_coal = t_ref + t0 (Sec. II: t0 ~ 1 yr) */
    int device;             /* CUDA device ordinal */
    void *stream;           /* cudaStream_t to run on; NULL = the library creates one */
    int max_batch;          /* largest B any call will use (device buffers sized for it) */
    double timeout_s;       /* bound on host waits for the device; <= 0 means 60 s */
} lisa_like_config;

/* Fill *cfg with the defaults: six modes, K = 1024, FP64, t0 = 1 yr, device 0. */
void lisa_like_default_config(lisa_like_config *cfg);

/* Create a handle (Sec. II.A: everything that is done once before > 1e7 calls).
 * Errors: LISA_ERR_ARG for a bad config, LISA_ERR_CUDA / LISA_ERR_OOM. */
lisa_status lisa_like_create(const lisa_like_config *cfg, lisa_like_t **out);

/* Upload the data stream and PSD once (Sec. II.A; the PSD of Sec. II).
 *   f0 > 0, df > 0: the grid f_j = f0 + j df, j = 0 .. n_bins-1, 1 <= n_bins < 2^31.
 *   d   host double[3][n_bins][2], the A, E, T data d~(f_j); NULL means d = 0.
 *   psd host double[3][n_bins], one-sided S_n^{A,E,T}(f_j) > 0 and finite.
 * Stores w = 4 df / S and w d on the device and computes <d|d> (FP64).
 * Errors: LISA_ERR_ARG (NULL psd, non-finite value, S <= 0, bad grid). */
lisa_status lisa_like_set_data(lisa_like_t *h, double f0, double df, int64_t n_bins,
                               const double *d, const double *psd);

/* Batched ln L for B host parameter rows (1 <= B <= max_batch); blocks until done.
 *   params host double[B][11]; lnL host double[B]; dh, hh host double[B] or NULL.
 * Errors: LISA_ERR_STATE before set_data, LISA_ERR_ARG, LISA_ERR_CUDA,
 * LISA_ERR_TIMEOUT when the device does not finish within the configured bound. */
lisa_status lisa_like_loglike(lisa_like_t *h, const double *params, int B, double *lnL,
                              double *dh, double *hh);

/* Same on device pointers, asynchronous on `stream` (a cudaStream_t; NULL is CUDA's
 * default stream, as everywhere in CUDA).
 *   d_params device double[B][11]; d_lnL device double[B]; d_dh, d_hh device or NULL.
 * The call returns after enqueueing; the caller synchronises the stream.  Calls on one
 * handle share its work buffers: do not overlap two of them on different streams. */
lisa_status lisa_like_loglike_device(lisa_like_t *h, const double *d_params, int B,
                                     double *d_lnL, double *d_dh, double *d_hh, void *stream);

/* <d|d> of the uploaded data (Eqs. (3), (11)). */
lisa_status lisa_like_data_inner(const lisa_like_t *h, double *dd);

/* Dense template of one walker on the uploaded grid, materialised (for making
 * injections and for element-wise checks): out host double[3][n_bins][2]. */
lisa_status lisa_like_template(lisa_like_t *h, const double *params, double *out);

/* Intermediate results of steps 1-2 for B host walkers, copied to host buffers:
 *   band  int64_t[B][n_modes][3]: active flag, j_lo, j_hi (inclusive dense-bin range)
 *   fedge double[B][n_modes][2]: f_lo, f_hi [Hz]
 *   fk    double[B][n_modes][K]: knot frequencies
 *   vals  double[B][n_modes][8][K]: A, phase (+ delay phase), Re/Im T^A, T^E, T^T
 * Any output may be NULL. Requires set_data (the grid sets the bands). */
lisa_status lisa_like_stage_knots(lisa_like_t *h, const double *params, int B, int64_t *band,
                                  double *fedge, double *fk, double *vals);

/* Spline coefficients of step 3 for B host walkers:
 *   coef double[B][n_modes][K-1][8][4]; segment s, series q: c0 + c1 x + c2 x^2 + c3 x^3
 *   with x = f - f_s. Requires set_data. */
lisa_status lisa_like_stage_coeffs(lisa_like_t *h, const double *params, int B, double *coef);

/* Luminosity distance [Gpc] at redshift z (flat LambdaCDM, H0 = 67.7, Om = 0.31),
 * host-side helper for turning the redshifts of a workload into D_L. NaN if z < 0. */
double lisa_dl_from_z(double z);

/* Stand-in one-sided A/E/T PSD at f_j = f0 + j df, host helper: out host
 * double[3][n_bins]. Returns LISA_ERR_ARG for a bad grid. */
lisa_status lisa_psd_aet(double f0, double df, int64_t n_bins, double *out);

/* Per-stage device timing with CUDA events (on = 1) of subsequent loglike and
 * loglike_device calls, recorded on the stream each call runs on. */
lisa_status lisa_like_set_profiling(lisa_like_t *h, int on);

/* Sums of the per-stage device times [ms] of the calls profiled since the last read,
 * ms[0] knots, ms[1] splines, ms[2] split-precision segment preparation (0 in FP64),
 * ms[3] work planning, ms[4] fused dense ln L, ms[5] finishing (ms holds 6 doubles);
 * *n_calls receives the number of calls summed.  Waits (bounded by the configured
 * timeout) for those calls, then clears the sums. */
lisa_status lisa_like_read_profile(lisa_like_t *h, double *ms, int *n_calls);

/* Limits of lisa_like_loglike_noalloc and the size of its static scratch. */
#define LISA_NOALLOC_SCRATCH_BYTES 4194304
#define LISA_NOALLOC_MAX_WALKER_MODE_KNOTS 8192
#define LISA_NOALLOC_MAX_ITEMS 16384

/* Batched ln L that allocates no memory (the paper has no counterpart: this entry
 * exists for callers that cannot call cudaMalloc, e.g. code inside a framework that
 * owns the whole device heap and gives an operation only its buffers, or a real-time
 * loop that cannot afford the device synchronisation an allocation implies).  It needs
 * no handle; the caller passes every input and output as device memory, and all
 * per-call scratch lives in one static device array of LISA_NOALLOC_SCRATCH_BYTES
 * inside this library, which every GPU that loads the library holds until exit.
 *   cfg          n_modes, modes, n_knots and t0_s are used; the other fields ignored.
 *   f0, df, n_bins  the grid f_j = f0 + j df (as for set_data).
 *   d_bins       device double[n_bins][9], per bin: w_A, w_E, w_T, then (w d)_A re,
 *                im, (w d)_E re, im, (w d)_T re, im, with w = 4 df / S_n (Eq. (3));
 *                16-byte aligned (as cudaMalloc and torch allocations are).
 *   dd           <d|d> of those data (host value; enters ln L only as -dd/2).
 *   d_params     device double[B][11]; d_lnL device double[B]; d_dh, d_hh device
 *                double[B] or NULL.
 *   stream       cudaStream_t (NULL = CUDA's default stream); the call only enqueues.
 * Limits: B * n_modes * n_knots <= LISA_NOALLOC_MAX_WALKER_MODE_KNOTS and
 * B * (ceil(n_bins / 1024) + 1) <= LISA_NOALLOC_MAX_ITEMS; larger requests return
 * LISA_ERR_ARG, and lisa_like_last_error(NULL) on the same thread says which limit.
 * The first call on a device looks up the scratch address on that device (with it
 * current), so make that first call before any stream capture.  The address is kept
 * for the life of the process: resetting a device (cudaDeviceReset) or re-creating its
 * primary context after the first call is not supported.  Every call shares the
 * one scratch array and leaves its contents behind: calls that overlap on the GPU
 * (different streams or host threads) race and must be serialised by the caller. */
lisa_status lisa_like_loglike_noalloc(const lisa_like_config *cfg, double f0, double df,
                                      int64_t n_bins, const double *d_bins, double dd,
                                      const double *d_params, int B, double *d_lnL,
                                      double *d_dh, double *d_hh, void *stream);

/* Test of the device-side timeout path (the paper has no counterpart).  With polls > 0
 * the dense kernels of later calls on this handle arm each data tile's barrier for the
 * tile's bytes but issue no copy, so every wait on it gives up after `polls` polls with
 * no copy in flight: the call then returns LISA_ERR_TIMEOUT (loglike) or NaN outputs
 * (loglike_device), exactly as when a real staging copy never completes.  polls = 0
 * restores normal operation.  Errors: LISA_ERR_ARG for polls outside [0, 2^20]. */
lisa_status lisa_like_test_device_wait(lisa_like_t *h, int polls);

/* Capture the whole per-call kernel sequence in a CUDA graph (on = 1) and replay it.
 * The executable is cached for the last (B, parameter and output pointers) and
 * rebuilt when they change; it runs on the handle's stream, ordered after and before
 * the caller's stream by events.  Per-stage profiling does not apply to graph
 * replays. */
lisa_status lisa_like_set_graphs(lisa_like_t *h, int on);

/* Tile shape of the fused dense kernel: `per_thread` consecutive bins per thread (the
 * tile is 128 x per_thread bins) and `group` walkers sharing one staged data tile.
 * Supported: (8,8), (4,8), (16,8) in split precision only, (8,1).  LISA_ERR_ARG
 * otherwise.  out[3] of get_tune: per_thread, group, persistent blocks. */
lisa_status lisa_like_set_tune(lisa_like_t *h, int per_thread, int group);
lisa_status lisa_like_get_tune(const lisa_like_t *h, int *out);

/* Autotuner: times every supported tile shape on the full call for these B host
 * walkers (a representative sample is enough), keeps the fastest, and caches the
 * choice per (n_bins, n_knots, precision) in the handle; later calls with the same
 * key reuse it without timing.  out[3] (or NULL) receives the chosen shape.
 * Requires set_data. */
lisa_status lisa_like_autotune(lisa_like_t *h, const double *params, int B, int *out);

/* Per-mode inner products, each mode's template alone (no cross terms): for walker b
 * and mode i (the config's order), dh_modes[b][i] = <d|h_i> and hh_modes[b][i] =
 * <h_i|h_i>, the per-harmonic SNR^2 of Table III computed "in isolation".  Because
 * the template is a sum over modes, sum_i <d|h_i> = <d|h> of loglike.  Host buffers
 * double[B][n_modes] (either may be NULL); blocks until done. */
lisa_status lisa_like_mode_inner(lisa_like_t *h, const double *params, int B, double *dh_modes,
                                 double *hh_modes);

/* Number of kernel launches the last loglike / loglike_device call enqueued. */
int lisa_like_last_launches(const lisa_like_t *h);

/* Release every resource of the handle (NULL is allowed). */
void lisa_like_destroy(lisa_like_t *h);

/* Human-readable description of the last failure on this handle ("" if none);
 * with h == NULL, the last failure of lisa_like_create or lisa_like_loglike_noalloc
 * on this thread. */
const char *lisa_like_last_error(const lisa_like_t *h);

/* The mode-pair inner products Re<h_lm|h_l'm'> of B walkers (host params [B][11]),
 * cross [B][L][L] (host, symmetric; the diagonal is <h_lm|h_lm>).  With the per-mode
 * <d|h_lm> of lisa_like_mode_inner, ln L = sum_lm <d|h_lm> - 1/2 sum <h_lm|h_l'm'>
 * - <d|d>/2: the mode-by-mode form with cross terms that the paper contrasts with its
 * single combined data stream (Sec. II.A), and the reason the total SNR of Table III is
 * not the quadrature sum of the mode SNRs.  Computed from the template of every mode
 * and mode pair: Re<h_a|h_b> = (<h_a + h_b|h_a + h_b> - <h_a|h_a> - <h_b|h_b>) / 2
 * (L (L + 1) / 2 likelihood passes).  Blocking. */
lisa_status lisa_like_mode_cross(lisa_like_t *h, const double *params, int B, double *cross);

/* ------------------------------------------------------------------ relative binning
 * A cheaper approximation of the same ln L, which the paper leaves as future work
 * (Sec. II.A): relative binning (Zackay, Dai & Venumadhav 2018), the heterodyning of
 * Cornish (2010).  A fiducial waveform h0 (parameters near the posterior) fixes coarse
 * bins -- n_rb + 1 edges log-spaced in frequency over the union of its mode bands,
 * snapped to the grid, plus every mode's band start and end + 1 -- and per-bin summary
 * data of every mode lm, channel c and bin b (w = 4 df / S, Eq. (3)):
 *   A0 = sum w d h0_lm*,  A1 = sum w d h0_lm* (f - f_b),
 *   B0 = sum w h0_lm h0_l'm'*,  B1 = sum w h0_lm h0_l'm'* (f - f_b)  (mode pairs).
 * A template's modes are then evaluated only at the edges (waveform and response at each
 * edge frequency, no spline); their ratios to h0 are linear across each bin (held
 * constant across a bin where h0 vanishes at one edge), and <d|h>, <h|h>, ln L follow from
 * the summary data.  Exact at the fiducial and for templates whose ratio to it is
 * constant; the error grows as the square of the bin width.
 *
 * lisa_like_set_fiducial: summary data for `params` [11] (host) with n_rb in [8, 256]
 * coarse bins, on the data of the last lisa_like_set_data (set_data discards them).
 * Synchronous.  Errors: LISA_ERR_STATE without data, LISA_ERR_ARG for invalid
 * parameters or a fiducial with no active mode. */
lisa_status lisa_like_set_fiducial(lisa_like_t *h, const double *params, int n_rb);

/* The bin edges as grid indices (edges may be NULL to query *n_edges). */
lisa_status lisa_like_rb_edges(lisa_like_t *h, int64_t *edges, int *n_edges);

/* ln L, <d|h>, <h|h> by relative binning for B walkers (host buffers, blocking; dh, hh may
 * be NULL).  Invalid walkers: -inf, 0, 0. */
lisa_status lisa_like_loglike_rb(lisa_like_t *h, const double *params, int B, double *lnL,
                                 double *dh, double *hh);
/* The same on device pointers, enqueued on `stream` (NULL = default stream). */
lisa_status lisa_like_loglike_rb_device(lisa_like_t *h, const double *d_params, int B,
                                        double *d_lnL, double *d_dh, double *d_hh, void *stream);

#ifdef __cplusplus
}
#endif
#endif
