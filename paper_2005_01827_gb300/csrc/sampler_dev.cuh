// sampler_dev.cuh -- device helpers shared by the sampler and flow kernels: the
// Philox4x32-10 generator, uniforms, the prior box, the Gaussian test target and the
// conversion of sampling coordinates to physical parameters (internal header).
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/lisa_sampler.h"

namespace lisa_smp {

constexpr int D = LISA_SAMPLER_NDIM;
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kYearS = 3.15576e7;                  // orbital period of the constellation
constexpr double kAuS = 1.495978707e11 / 299792458.0;  // 1 AU in light seconds

// ------------------------------------------------------------------ Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror & Shaw (2011): ten rounds of two
// 32x32 -> 64-bit products with the Weyl key schedule.
__host__ __device__ inline uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

struct U4 {
    uint32_t v[4];
};

__host__ __device__ inline U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; r++) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = mulhi32(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = mulhi32(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    U4 o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}

// uniform in (0, 1): (u + 1/2) 2^-32, exact in FP64
__host__ __device__ inline double unit(uint32_t u) { return ((double)u + 0.5) * 0x1p-32; }

__device__ inline double ln_prior(const double *x, const double *lo, const double *hi) {
    for (int q = 0; q < D; q++)
        if (!(x[q] >= lo[q] && x[q] <= hi[q])) return -INFINITY;
    return 0.0;
}

// Gaussian test target, every operation rounded as written
__device__ inline double gauss_lnl(const double *x, const double *mean, const double *sig) {
    double acc = 0.0;
    for (int q = 0; q < D; q++) {
        const double r = __ddiv_rn(__dsub_rn(x[q], mean[q]), sig[q]);
        acc = __dadd_rn(acc, __dmul_rn(r, r));
    }
    return __dmul_rn(-0.5, acc);
}

// LISA frame -> SSB frame.  The constellation of the response model is a fixed triangle
// rotated by Q = Rz(alpha) Ry(-pi/3) Rz(-alpha), alpha = 2 pi t / yr; the LISA frame is
// the one in which the triangle is at rest, at the arrival time t_L (absolute seconds).
__device__ inline void lisa_to_ssb(double tL, double lamL, double betL, double psiL, double *t,
                                   double *lam, double *bet, double *psi) {
    double sa, ca;
    sincos(2.0 * kPi * tL / kYearS, &sa, &ca);
    const double h = 0.8660254037844386467637231707529362;  // sqrt(3)/2
    const double Q[3][3] = {{0.5 * ca * ca + sa * sa, -0.5 * ca * sa, -h * ca},
                            {-0.5 * ca * sa, 0.5 * sa * sa + ca * ca, -h * sa},
                            {h * ca, h * sa, 0.5}};
    double sl, cl, sb, cb, sp, cp;
    sincos(lamL, &sl, &cl);
    sincos(betL, &sb, &cb);
    sincos(psiL, &sp, &cp);
    // direction to the source and polarisation axis cos(psi) u + sin(psi) v in the L frame
    const double nL[3] = {cb * cl, cb * sl, sb};
    const double pL[3] = {cp * sl - sp * sb * cl, -cp * cl - sp * sb * sl, sp * cb};
    double n[3], p[3];
    for (int i = 0; i < 3; i++) {
        n[i] = Q[i][0] * nL[0] + Q[i][1] * nL[1] + Q[i][2] * nL[2];
        p[i] = Q[i][0] * pL[0] + Q[i][1] * pL[1] + Q[i][2] * pL[2];
    }
    double l = atan2(n[1], n[0]);
    if (l < 0.0) l += 2.0 * kPi;
    const double nz = fmin(1.0, fmax(-1.0, n[2]));
    // u = (n_y, -n_x, 0)/rho and v = (-n_z n_x, -n_z n_y, rho^2)/rho with rho = cos(beta)
    const double rho2 = n[0] * n[0] + n[1] * n[1];
    double ps = atan2(-nz * (p[0] * n[0] + p[1] * n[1]) + p[2] * rho2, p[0] * n[1] - p[1] * n[0]);
    ps = fmod(ps, kPi);
    if (ps < 0.0) ps += kPi;
    // arrival at the centre t_L = t + k . p0(t) with k = -n: fixed point in t
    double tt = tL;
    for (int it = 0; it < 6; it++) {
        double s2, c2;
        sincos(2.0 * kPi * tt / kYearS, &s2, &c2);
        tt = tL + kAuS * (n[0] * c2 + n[1] * s2);
    }
    *t = tt;
    *lam = l;
    *bet = asin(nz);
    *psi = ps;
}

// sampling coordinates of Table I -> physical parameters of the likelihood
__device__ inline void to_physical(const double *x, int lisa_frame, double t0, double *th) {
    th[0] = exp(x[0]);
    th[1] = x[1];
    th[2] = x[2];
    th[3] = x[3];
    th[4] = exp(x[4]);
    th[5] = x[5];
    th[6] = acos(x[6]);
    if (lisa_frame) {
        double t, l, b, p;
        lisa_to_ssb(exp(x[10]) + t0, x[7], asin(x[8]), x[9], &t, &l, &b, &p);
        th[7] = l;
        th[8] = b;
        th[9] = p;
        th[10] = t - t0;
    } else {
        th[7] = x[7];
        th[8] = asin(x[8]);
        th[9] = x[9];
        th[10] = exp(x[10]);
    }
}

// parameters the likelihood rejects (lnL = -inf, no dense work)
__device__ inline void invalid_params(double *th) {
    th[0] = __longlong_as_double(0x7ff8000000000000LL);
    for (int q = 1; q < D; q++) th[q] = 0.0;
}


}  // namespace lisa_smp
