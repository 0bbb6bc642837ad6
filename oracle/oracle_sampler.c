/*
 * oracle_sampler.c -- plain CPU reference of the parallel-tempered affine-invariant
 * ensemble sampler of Sec. III.  TEST INFRASTRUCTURE ONLY: nothing in the product
 * library links or calls it, and it shares no code with the CUDA path.
 *
 *  - Stretch move (Sec. III.A): the ensemble of one temperature is split into two
 *    halves; every walker k of the active half takes a partner j drawn uniformly from
 *    the other half and a scale y from g(y) ~ 1/sqrt(y) on [1/a, a] (Eq. (15)); the
 *    proposal x_j + y (x_k - x_j) of Eq. (14) is accepted with probability
 *    min(1, y^(D-1) [L(new)/L(old)]^beta pi(new)/pi(old)), Eq. (16) with the tempered
 *    likelihood of Sec. III.B and the prior ratio.
 *  - Parallel tempering (Sec. III.B): after both halves, walker w of temperature t and
 *    walker w of temperature t+1 exchange states with probability
 *    min(1, [L_{t+1}/L_t]^(beta_t - beta_{t+1})) (Eq. (17)), pairs taken from the
 *    hottest down to the coldest.
 *  - Adaptive ladder (Vousden, Farr & Mandel 2016): the log temperature gaps
 *    S_g = ln(T_{g+1} - T_g) move by kappa(s) (A_g - A_{g+1}) after each step s, with
 *    A_g the fraction of accepted swaps between temperatures g and g+1 in that step and
 *    kappa(s) = t0 / (nu (s + t0)); the coldest and the hottest temperature stay fixed.
 *  - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011); counter
 *    (step, phase, temperature, walker) with phase 0/1 for the two halves and 2 for the
 *    swaps, key = the 64-bit seed; uniforms (u32 + 0.5) / 2^32.
 *  - Coordinates (Table I): x = (ln M_T, q, a1, a2, ln D_L, phi_ref, cos iota, lambda,
 *    sin beta, psi, ln t_ref) with a uniform prior inside [lower, upper].  With the
 *    LISA-frame option (Sec. II: sampled in the LISA frame, converted before waveform
 *    generation), lambda, beta, psi and t_ref are LISA-frame values.
 *  - LISA frame (stand-in, tied to the rigid constellation of the response model): the
 *    orthonormal frame in which the three spacecraft stay fixed, at the arrival time of
 *    the signal at the constellation centre.  The constellation of the response model is
 *    the fixed triangle rotated by Q(t) = Rz(alpha) Ry(-pi/3) Rz(-alpha), with
 *    alpha = 2 pi t / yr, so the LISA-frame direction n_L maps to Q n_L.  The time of
 *    arrival at the centre is t_L = t_SSB + k . p0(t_SSB) (k the propagation direction,
 *    p0 the centre in light seconds).
 *  - Autocorrelation time (Sec. III.C): normalised autocorrelation per walker with the
 *    1/(N - tau) estimator of Eqs. (19)-(21), averaged over walkers; Eq. (22)
 *    tau(M) = 1 + 2 sum_{t=1}^M rho(t) at the smallest M with M >= 5 tau(M).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define NDIM 11
#define PI_D 3.14159265358979323846
#define YEAR_SEC 31557600.0
#define AU_SEC (1.495978707e11 / 299792458.0)

/* ------------------------------------------------------------------ Philox4x32-10 */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k[0];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k[1];
    c[1] = (uint32_t)p1;
    c[3] = (uint32_t)p0;
    c[0] = n0;
    c[2] = n2;
}

void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; r++) {
        if (r > 0) { /* Weyl key schedule */
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof(c));
}

static void draws(uint64_t seed, uint32_t step, uint32_t phase, uint32_t t, uint32_t w,
                  double u[4])
{
    const uint32_t ctr[4] = {step, phase, t, w};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    oracle_philox(ctr, key, o);
    for (int i = 0; i < 4; i++) u[i] = ((double)o[i] + 0.5) * (1.0 / 4294967296.0);
}

/* ------------------------------------------------------------------ LISA frame */
static void rot_q(double alpha, double Q[3][3])
{
    /* Q = Rz(alpha) Ry(-pi/3) Rz(-alpha) */
    const double ca = cos(alpha), sa = sin(alpha);
    const double ct = 0.5, st = -sqrt(3.0) / 2.0;
    const double Rz[3][3] = {{ca, -sa, 0.0}, {sa, ca, 0.0}, {0.0, 0.0, 1.0}};
    const double Ry[3][3] = {{ct, 0.0, st}, {0.0, 1.0, 0.0}, {-st, 0.0, ct}};
    const double Rzi[3][3] = {{ca, sa, 0.0}, {-sa, ca, 0.0}, {0.0, 0.0, 1.0}};
    double M[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            M[i][j] = 0.0;
            for (int k = 0; k < 3; k++) M[i][j] += Ry[i][k] * Rzi[k][j];
        }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            Q[i][j] = 0.0;
            for (int k = 0; k < 3; k++) Q[i][j] += Rz[i][k] * M[k][j];
        }
}

/* unit direction to the source and the polarisation axis p = cos psi u + sin psi v */
static void sky_vectors(double lam, double beta, double psi, double n[3], double p[3])
{
    const double cl = cos(lam), sl = sin(lam), cb = cos(beta), sb = sin(beta);
    const double u[3] = {sl, -cl, 0.0};
    const double v[3] = {-sb * cl, -sb * sl, cb};
    n[0] = cb * cl;
    n[1] = cb * sl;
    n[2] = sb;
    for (int i = 0; i < 3; i++) p[i] = cos(psi) * u[i] + sin(psi) * v[i];
}

static void sky_angles(const double n[3], const double p[3], double *lam, double *beta,
                       double *psi)
{
    double l = atan2(n[1], n[0]);
    if (l < 0.0) l += 2.0 * PI_D;
    double z = n[2];
    if (z > 1.0) z = 1.0;
    if (z < -1.0) z = -1.0;
    const double b = asin(z);
    const double cl = cos(l), sl = sin(l), cb = cos(b), sb = sin(b);
    const double u[3] = {sl, -cl, 0.0};
    const double v[3] = {-sb * cl, -sb * sl, cb};
    double ps = atan2(p[0] * v[0] + p[1] * v[1] + p[2] * v[2],
                      p[0] * u[0] + p[1] * u[1] + p[2] * u[2]);
    ps = fmod(ps, PI_D);
    if (ps < 0.0) ps += PI_D;
    *lam = l;
    *beta = b;
    *psi = ps;
}

static double kdotp0(const double n[3], double t)
{
    /* propagation direction k = -n; centre p0 on the 1-AU circle */
    const double al = 2.0 * PI_D * t / YEAR_SEC;
    return -(n[0] * AU_SEC * cos(al) + n[1] * AU_SEC * sin(al));
}

/* (t_L, lambda_L, beta_L, psi_L) -> (t_SSB, lambda, beta, psi); times absolute [s] */
void oracle_lisa_to_ssb(const double *in, double *out)
{
    double Q[3][3], nL[3], pL[3], n[3], p[3];
    rot_q(2.0 * PI_D * in[0] / YEAR_SEC, Q);
    sky_vectors(in[1], in[2], in[3], nL, pL);
    for (int i = 0; i < 3; i++) {
        n[i] = Q[i][0] * nL[0] + Q[i][1] * nL[1] + Q[i][2] * nL[2];
        p[i] = Q[i][0] * pL[0] + Q[i][1] * pL[1] + Q[i][2] * pL[2];
    }
    sky_angles(n, p, &out[1], &out[2], &out[3]);
    double t = in[0];
    for (int it = 0; it < 6; it++) t = in[0] - kdotp0(n, t);
    out[0] = t;
}

/* inverse of oracle_lisa_to_ssb */
void oracle_ssb_to_lisa(const double *in, double *out)
{
    double Q[3][3], n[3], p[3], nL[3], pL[3];
    sky_vectors(in[1], in[2], in[3], n, p);
    const double tL = in[0] + kdotp0(n, in[0]);
    rot_q(2.0 * PI_D * tL / YEAR_SEC, Q);
    for (int i = 0; i < 3; i++) {
        nL[i] = Q[0][i] * n[0] + Q[1][i] * n[1] + Q[2][i] * n[2];
        pL[i] = Q[0][i] * p[0] + Q[1][i] * p[1] + Q[2][i] * p[2];
    }
    sky_angles(nL, pL, &out[1], &out[2], &out[3]);
    out[0] = tL;
}

/* physical parameters of the likelihood from the sampling coordinates */
void oracle_to_physical(const double *x, int lisa_frame, double t0, double *th)
{
    th[0] = exp(x[0]);
    th[1] = x[1];
    th[2] = x[2];
    th[3] = x[3];
    th[4] = exp(x[4]);
    th[5] = x[5];
    th[6] = acos(x[6]);
    if (lisa_frame) {
        const double in[4] = {exp(x[10]) + t0, x[7], asin(x[8]), x[9]};
        double o[4];
        oracle_lisa_to_ssb(in, o);
        th[7] = o[1];
        th[8] = o[2];
        th[9] = o[3];
        th[10] = o[0] - t0;
    } else {
        th[7] = x[7];
        th[8] = asin(x[8]);
        th[9] = x[9];
        th[10] = exp(x[10]);
    }
}

/* ------------------------------------------------------------------ ladder */
void oracle_default_ladder(int T, double ratio, int t_max_inf, double *betas)
{
    /* geometric temperatures 1, r, r^2, ... (Sec. III.B); optionally the hottest infinite */
    for (int t = 0; t < T; t++) betas[t] = 1.0 / pow(ratio, (double)t);
    if (t_max_inf && T > 1) betas[T - 1] = 0.0;
}

void oracle_adapt_ladder(int T, double *betas, const double *A, double kappa)
{
    if (T < 3) return;
    double *gap = malloc(sizeof(double) * T);
    for (int g = 0; g + 1 < T - 1; g++) {
        const double dS = kappa * (A[g] - A[g + 1]);
        gap[g] = (1.0 / betas[g + 1] - 1.0 / betas[g]) * exp(dS);
    }
    double Tacc = 1.0 / betas[0];
    for (int g = 0; g + 1 < T - 1; g++) {
        Tacc += gap[g];
        betas[g + 1] = 1.0 / Tacc;
    }
    free(gap);
}

/* ------------------------------------------------------------------ targets */
static double ln_prior(const double *x, const double *lo, const double *hi)
{
    for (int i = 0; i < NDIM; i++)
        if (!(x[i] >= lo[i] && x[i] <= hi[i])) return -INFINITY;
    return 0.0;
}

typedef struct {
    int kind; /* 0 Gaussian, 1 LISA likelihood */
    const double *mean, *sigma;
    double t0, f0, df;
    const int *modes;
    int n_modes, K, lisa_frame;
    int64_t n_bins;
    const double *d, *psd;
    int n_threads;
} target_t;

/* ln L of n points; points outside the prior get -inf without evaluation */
static void target_lnl(const target_t *tg, const double *x, const double *lnp, int n, double *out)
{
    if (tg->kind == 0) {
        for (int i = 0; i < n; i++) {
            double s = 0.0;
            for (int q = 0; q < NDIM; q++) {
                const double r = (x[NDIM * i + q] - tg->mean[q]) / tg->sigma[q];
                s += r * r;
            }
            out[i] = -0.5 * s;
        }
        return;
    }
    double *th = malloc(sizeof(double) * NDIM * (size_t)(n > 0 ? n : 1));
    double *lv = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int *idx = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int m = 0;
    for (int i = 0; i < n; i++) {
        out[i] = -INFINITY;
        if (isfinite(lnp[i])) {
            oracle_to_physical(x + NDIM * i, tg->lisa_frame, tg->t0, th + NDIM * m);
            idx[m++] = i;
        }
    }
    if (m > 0) {
        oracle_loglike(th, m, tg->t0, tg->modes, tg->n_modes, tg->K, tg->f0, tg->df, tg->n_bins,
                       tg->d, tg->psd, tg->n_threads, lv, NULL, NULL, NULL);
        for (int i = 0; i < m; i++) out[idx[i]] = lv[i];
    }
    free(th);
    free(lv);
    free(idx);
}

/* ------------------------------------------------------------------ sampler */
static int run(const target_t *tg, const oracle_sampler_cfg *c, int step0, int n_steps,
               double *x, double *lnl, double *chain, double *lnl_chain, long long *acc,
               long long *swaps)
{
    const int T = c->T, W = c->W;
    if (T < 1 || W < 4 || (W & 1) || !(c->a > 1.0)) return 0;
    const int H = W / 2;
    double *betas = c->betas;
    double *lnp = malloc(sizeof(double) * T * W);
    double *y = malloc(sizeof(double) * NDIM * T * H);
    double *ly = malloc(sizeof(double) * T * H), *py = malloc(sizeof(double) * T * H);
    double *zz = malloc(sizeof(double) * T * H);
    double *A = malloc(sizeof(double) * T);
    for (int i = 0; i < T * W; i++) lnp[i] = ln_prior(x + NDIM * i, c->lower, c->upper);
    target_lnl(tg, x, lnp, T * W, lnl);
    for (int s = 0; s < n_steps; s++) {
        const uint32_t step = (uint32_t)(step0 + s);
        for (int h = 0; h < 2; h++) {
            /* proposals for the active half h against the other half */
            for (int t = 0; t < T; t++)
                for (int kk = 0; kk < H; kk++) {
                    const int k = h * H + kk, p = t * H + kk;
                    double u[4];
                    draws(c->seed, step, (uint32_t)h, (uint32_t)t, (uint32_t)k, u);
                    int jj = (int)(u[0] * H);
                    if (jj > H - 1) jj = H - 1;
                    const int j = (1 - h) * H + jj;
                    const double g = (c->a - 1.0) * u[1] + 1.0;
                    const double z = g * g / c->a; /* inverse CDF of g(y) ~ 1/sqrt(y) */
                    const double *xk = x + NDIM * (t * W + k), *xj = x + NDIM * (t * W + j);
                    double *yy = y + NDIM * p;
                    for (int q = 0; q < NDIM; q++) yy[q] = xj[q] + z * (xk[q] - xj[q]);
                    zz[p] = z;
                    py[p] = ln_prior(yy, c->lower, c->upper);
                }
            target_lnl(tg, y, py, T * H, ly);
            for (int t = 0; t < T; t++)
                for (int kk = 0; kk < H; kk++) {
                    const int k = h * H + kk, i = t * W + k, p = t * H + kk;
                    double u[4];
                    draws(c->seed, step, (uint32_t)h, (uint32_t)t, (uint32_t)k, u);
                    double lr = (double)(NDIM - 1) * log(zz[p]) + py[p] - lnp[i];
                    if (betas[t] > 0.0) lr += betas[t] * (ly[p] - lnl[i]);
                    acc[2 * t + 1]++;
                    if (isfinite(py[p]) && log(u[2]) < lr) {
                        memcpy(x + NDIM * i, y + NDIM * p, sizeof(double) * NDIM);
                        lnl[i] = ly[p];
                        lnp[i] = py[p];
                        acc[2 * t]++;
                    }
                }
        }
        /* temperature swaps, hottest pair first */
        for (int t = 0; t < T; t++) A[t] = 0.0;
        for (int t = T - 2; t >= 0; t--) {
            int n_acc = 0;
            for (int w = 0; w < W; w++) {
                double u[4];
                draws(c->seed, step, 2u, (uint32_t)t, (uint32_t)w, u);
                const int i = t * W + w, j = (t + 1) * W + w;
                const double la = (betas[t] - betas[t + 1]) * (lnl[j] - lnl[i]);
                if (log(u[0]) < la) {
                    double tmp[NDIM];
                    memcpy(tmp, x + NDIM * i, sizeof(tmp));
                    memcpy(x + NDIM * i, x + NDIM * j, sizeof(tmp));
                    memcpy(x + NDIM * j, tmp, sizeof(tmp));
                    double v = lnl[i];
                    lnl[i] = lnl[j];
                    lnl[j] = v;
                    v = lnp[i];
                    lnp[i] = lnp[j];
                    lnp[j] = v;
                    n_acc++;
                }
            }
            swaps[2 * t] += n_acc;
            swaps[2 * t + 1] += W;
            A[t] = (double)n_acc / (double)W;
        }
        if (c->adaptive)
            oracle_adapt_ladder(T, betas, A,
                                c->adapt_lag / (c->adapt_time * ((double)step + c->adapt_lag)));
        if (chain) memcpy(chain + (size_t)NDIM * W * s, x, sizeof(double) * NDIM * W);
        if (lnl_chain) memcpy(lnl_chain + (size_t)W * s, lnl, sizeof(double) * W);
    }
    free(lnp);
    free(y);
    free(ly);
    free(py);
    free(zz);
    free(A);
    return 1;
}

int oracle_sampler_gauss(const oracle_sampler_cfg *c, const double *mean, const double *sigma,
                         int step0, int n_steps, double *x, double *lnl, double *chain,
                         double *lnl_chain, long long *acc, long long *swaps)
{
    target_t tg;
    memset(&tg, 0, sizeof(tg));
    tg.kind = 0;
    tg.mean = mean;
    tg.sigma = sigma;
    return run(&tg, c, step0, n_steps, x, lnl, chain, lnl_chain, acc, swaps);
}

int oracle_sampler_lisa(const oracle_sampler_cfg *c, double t0, const int *modes, int n_modes,
                        int K, double f0, double df, int64_t n_bins, const double *d,
                        const double *psd, int n_threads, int step0, int n_steps, double *x,
                        double *lnl, double *chain, double *lnl_chain, long long *acc,
                        long long *swaps)
{
    target_t tg;
    memset(&tg, 0, sizeof(tg));
    tg.kind = 1;
    tg.t0 = t0;
    tg.modes = modes;
    tg.n_modes = n_modes;
    tg.K = K;
    tg.lisa_frame = c->lisa_frame;
    tg.f0 = f0;
    tg.df = df;
    tg.n_bins = n_bins;
    tg.d = d;
    tg.psd = psd;
    tg.n_threads = n_threads;
    return run(&tg, c, step0, n_steps, x, lnl, chain, lnl_chain, acc, swaps);
}

/* Sec. III.C on one series per walker, chain[n][W].  The lags are taken one at a time,
 * each averaged over the walkers, until the window condition holds; rho_out [n] (may be
 * NULL) receives rho(0..M) and zeros beyond. */
double oracle_autocorr_time(const double *chain, int n, int W, double *rho_out)
{
    if (n < 2 || W < 1) return NAN;
    double *mu = calloc((size_t)W, sizeof(double)), *c0 = calloc((size_t)W, sizeof(double));
    int used = 0;
    for (int w = 0; w < W; w++) {
        for (int i = 0; i < n; i++) mu[w] += chain[(size_t)i * W + w];
        mu[w] /= n;
        for (int i = 0; i < n; i++) {
            const double v = chain[(size_t)i * W + w] - mu[w];
            c0[w] += v * v;
        }
        c0[w] /= n; /* Eq. (20) at lag 0 */
        if (c0[w] > 0.0) used++;
    }
    if (rho_out) memset(rho_out, 0, sizeof(double) * n);
    if (used == 0) {
        free(mu);
        free(c0);
        return NAN;
    }
    if (rho_out) rho_out[0] = 1.0;
    double tau = 1.0;
    for (int M = 1; M < n; M++) {
        double rho = 0.0; /* Eq. (19), averaged over the walkers */
        for (int w = 0; w < W; w++) {
            if (!(c0[w] > 0.0)) continue;
            double c = 0.0;
            for (int i = 0; i + M < n; i++)
                c += (chain[(size_t)i * W + w] - mu[w]) * (chain[(size_t)(i + M) * W + w] - mu[w]);
            rho += c / (double)(n - M) / c0[w];
        }
        rho /= used;
        if (rho_out) rho_out[M] = rho;
        tau += 2.0 * rho; /* Eq. (22) */
        if ((double)M >= 5.0 * tau) break;
    }
    free(mu);
    free(c0);
    return tau;
}
