/*
 * oracle.h -- plain FP64 CPU oracle for the batched LISA massive-black-hole-binary
 * log-likelihood of Katz, Marsat, Chua, Babak & Larson (2020).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls
 * this code; only tests/, __graft_entry__.smoke() and the cpu_baseline / reference
 * legs of bench.py use it.  It shares no source with the CUDA path.
 *
 * Parameter vector (Sec. II, the D = 11 list, in the paper's order):
 *   th[0]  M_T    total mass, detector frame [M_sun]
 *   th[1]  q      mass ratio m2/m1, 0 < q <= 1
 *   th[2]  a1     aligned dimensionless spin of the heavier hole, |a1| <= 0.99
 *   th[3]  a2     aligned dimensionless spin of the lighter hole, |a2| <= 0.99
 *   th[4]  D_L    luminosity distance [Gpc]
 *   th[5]  phi_ref reference phase [rad]
 *   th[6]  iota   inclination [rad]
 *   th[7]  lambda ecliptic longitude, SSB frame [rad]
 *   th[8]  beta   ecliptic latitude, SSB frame [rad]
 *   th[9]  psi    polarisation angle [rad]
 *   th[10] t_ref  reference time [s]; t_coal = t_ref + t0
 *
 * Mode order used by every array indexed by a mode: the (l,m) pairs are passed
 * explicitly as int modes[n_modes][2].
 *
 * Knot series order (8 real series per mode and knot):
 *   0 A, 1 phase (waveform phase + SSB-to-constellation delay phase),
 *   2 Re T^A, 3 Im T^A, 4 Re T^E, 5 Im T^E, 6 Re T^T, 7 Im T^T.
 *
 * Complex arrays are interleaved (re, im) doubles.  Channel arrays are [3][...]
 * in the order A, E, T.
 */
#ifndef LISA_ORACLE_H
#define LISA_ORACLE_H
#include <stdint.h>

#define ORACLE_NPAR 11
#define ORACLE_NSERIES 8

#ifdef __cplusplus
extern "C" {
#endif

/* spin-weighted spherical harmonic sY_lm(theta, phi) */
void oracle_sylm(int s, int l, int m, double theta, double phi, double *re, double *im);

/* (2,2)-mapped mode model at n frequencies: amplitude, phase, dphase/df, t_lm(f) */
int oracle_mode_eval(const double *th, double t0, int l, int m, const double *f, int64_t n,
                     double *amp, double *phase, double *dphase, double *tf);

/* peak frequency of f^2 A_22 [Hz] and the cut frequency of mode (l,m) [Hz] */
int oracle_peak_and_cut(const double *th, int l, int m, double *f_peak, double *f_cut);

/* spacecraft positions at time t [s]: centre p0[3], offsets q[3][3], in seconds */
void oracle_orbit(double t, double *p0, double *q);

/* TDI A,E,T transfer of mode (l,m) at (f[i], t[i]); T out [3][n][2] */
int oracle_transfer(const double *th, int l, int m, const double *f, const double *t, int64_t n,
                    double *T);

/* SSB-to-constellation-centre delay phase -2 pi f k.p0(t) */
double oracle_delay_phase(const double *th, double f, double t);

/* band of mode (l,m) on the grid; returns 1 when active, 0 when empty */
int oracle_band(const double *th, double t0, int l, int m, double f0, double df, int64_t n_bins,
                double *f_lo, double *f_hi, int64_t *j_lo, int64_t *j_hi);

/* knots and the 8 knot series of one mode; returns 1 when active */
int oracle_knots(const double *th, double t0, int l, int m, double f0, double df, int64_t n_bins,
                 int K, double *fk, double *vals /* [8][K] */);

/* not-a-knot cubic spline: c[(K-1)][4] with y = c0 + c1 x + c2 x^2 + c3 x^3, x = f - f_s */
int oracle_spline(int K, const double *x, const double *y, double *c);
/* evaluate a spline built by oracle_spline at n points using the segment rule */
void oracle_spline_eval(int K, const double *xk, const double *c, const double *f, int64_t n,
                        double *y);

/* dense template h[3][n_bins][2] by knots -> splines -> dense bins (Sec. II.A) */
int oracle_template(const double *th, double t0, const int *modes, int n_modes, int K,
                    double f0, double df, int64_t n_bins, double *h);
/* dense template by direct evaluation of waveform and response at every bin */
int oracle_direct(const double *th, double t0, const int *modes, int n_modes,
                  double f0, double df, int64_t n_bins, double *h);

/* one mode's A, E, T response at arbitrary frequencies (direct evaluation), zero outside
 * the mode's band on the grid; h [3][n][2] */
int oracle_mode_response(const double *th, double t0, int l, int m, double f0, double df,
                         int64_t n_bins, const double *f, int64_t n, double *h);

/* noise-weighted inner products of Eqs. (3) and (11): re<a|b> summed over A,E,T */
double oracle_inner(const double *a, const double *b, const double *psd, double df, int64_t n_bins);

/* batched log-likelihood Eq. (2) for B walkers; dh, hh, dd may be NULL */
int oracle_loglike(const double *th, int B, double t0, const int *modes, int n_modes, int K,
                   double f0, double df, int64_t n_bins, const double *d, const double *psd,
                   int n_threads, double *lnL, double *dh, double *hh, double *dd);

/* residual form -1/2 sum w |d-h|^2 for one walker (the second algebraic form of Eq. (2)) */
int oracle_loglike_residual(const double *th, double t0, const int *modes, int n_modes, int K,
                            double f0, double df, int64_t n_bins, const double *d,
                            const double *psd, double *lnL);

/* stand-in one-sided PSD of channels A,E,T at n frequencies; S[3][n] */
void oracle_psd_aet(const double *f, int64_t n, double *S);

/* coloured noise of Eq. (12): n[3][N][2] from white z[3][N][2] */
void oracle_noise(const double *psd, double df, int64_t n_bins, const double *z, double *noise);

/* luminosity distance [Gpc] at redshift z (flat LambdaCDM stand-in) */
double oracle_dl_gpc(double z);

/* plus/cross polarisations of one mode at positive f (reduced m>0 form), [n][2] each */
int oracle_polarizations(const double *th, double t0, int l, int m, const double *f, int64_t n,
                         double *hp, double *hc);

/* ---------------------------------------------------------------- sampler (Sec. III) */

/* Philox4x32-10 block: out = philox(ctr, key) */
void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* LISA-frame <-> SSB-frame sky position, polarisation and arrival time (Sec. II);
 * in/out = (t [s, absolute], lambda, beta, psi) */
void oracle_lisa_to_ssb(const double *in, double *out);
void oracle_ssb_to_lisa(const double *in, double *out);

/* physical parameters (header order above) from the sampling coordinates of Table I:
 * (ln M_T, q, a1, a2, ln D_L, phi_ref, cos iota, lambda, sin beta, psi, ln t_ref) */
void oracle_to_physical(const double *x, int lisa_frame, double t0, double *th);

/* geometric ladder beta_t = ratio^-t; the hottest beta = 0 when t_max_inf */
void oracle_default_ladder(int T, double ratio, int t_max_inf, double *betas);
/* one adaptive ladder update from the per-pair swap acceptances A[T-1] */
void oracle_adapt_ladder(int T, double *betas, const double *A, double kappa);

typedef struct {
    int T, W;              /* temperatures; walkers per temperature (even, >= 4) */
    double a;              /* stretch scale of Eq. (15) */
    double *betas;         /* [T] inverse temperatures, updated by the adaptive ladder */
    int adaptive;          /* Vousden et al. ladder adaptation */
    double adapt_lag, adapt_time;
    uint64_t seed;
    const double *lower, *upper; /* [11] uniform prior box */
    int lisa_frame;        /* lambda, beta, psi, t_ref sampled in the LISA frame */
} oracle_sampler_cfg;

/* n_steps of the PT stretch sampler on a Gaussian target (mean, sigma [11]) or on the
 * LISA likelihood; x [T][W][11] and lnl [T][W] are the state in/out; chain
 * [n_steps][W][11] and lnl_chain [n_steps][W] record the coldest temperature (may be
 * NULL); acc and swaps [T][2] accumulate (accepted, proposed). */
int oracle_sampler_gauss(const oracle_sampler_cfg *c, const double *mean, const double *sigma,
                         int step0, int n_steps, double *x, double *lnl, double *chain,
                         double *lnl_chain, long long *acc, long long *swaps);
int oracle_sampler_lisa(const oracle_sampler_cfg *c, double t0, const int *modes, int n_modes,
                        int K, double f0, double df, int64_t n_bins, const double *d,
                        const double *psd, int n_threads, int step0, int n_steps, double *x,
                        double *lnl, double *chain, double *lnl_chain, long long *acc,
                        long long *swaps);

/* autocorrelation time of Sec. III.C for chain[n][W]; rho_out [n] may be NULL */
double oracle_autocorr_time(const double *chain, int n, int W, double *rho_out);

#ifdef __cplusplus
}
#endif
#endif
