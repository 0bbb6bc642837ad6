// model.cuh -- device-side waveform, orbit and response model (Katz et al. 2020,
// Sec. II): the per-walker constants, the harmonic amplitude/phase of Eq. (5),
// t_lm(f) of Eq. (6) and the TDI A/E/T transfer of Eqs. (7)-(10).
//
// The fit coefficients the paper takes from PhenomHM and from the fast LISA
// response are stand-ins with the same functional form (marked STANDIN):
//   (2,2) phase: TaylorF2-type inspiral to 1.5PN below M f = 0.018, joined with
//     matching value, slope and curvature to a merger-ringdown a1 x - a2 / x form;
//   (2,2) amplitude: f^-7/6 with exp(alpha2 v^2 + alpha3 v^3), rolled off as
//     1 / (1 + (x / x_RD)^6) at the stand-in remnant ringdown frequency x_RD;
//   mode (l,m) at f: (2,2) model at 2 f / m (PhenomHM construction), amplitude
//     times a leading-order ratio, phase times m/2 plus a constant;
//   t_coal: time at the peak of f^2 A_22 (Sec. II);
//   orbit: rigid equal-arm cartwheel on a circular 1-AU orbit, arms 2.5 Gm;
//   link response: (-i pi f L) sinc(pi f L (1 - k.n)) e^{-i pi f (L + k.(q_s + q_r))},
//     first-generation X, Y, Z, and A, E, T of Eqs. (8)-(10).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace lisa {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTwoPi = 6.283185307179586476925286766559005768;
constexpr double kMsunS = 4.925490947641267e-06;  // G M_sun / c^3 [s]
constexpr double kClight = 299792458.0;
constexpr double kGpcM = 3.0856775814913673e25;
constexpr double kAuM = 1.495978707e11;
constexpr double kArmM = 2.5e9;
constexpr double kYearS = 3.15576e7;   // STANDIN orbital period
constexpr double kXJoin = 0.018;       // STANDIN inspiral / merger-ringdown join (M f)
constexpr double kXCut = 0.2;          // STANDIN cut of the (2,2)-mapped frequency (M f)
constexpr int kNPar = 11;
constexpr int kNSeries = 8;
constexpr int kMaxModes = 6;

struct cplx {
    double re, im;
};
__host__ __device__ inline cplx cmul(cplx a, cplx b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ inline cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ inline cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ inline cplx cscale(cplx a, double s) { return {a.re * s, a.im * s}; }
__device__ inline cplx cexpi(double ph) {
    double s, c;
    sincos(ph, &s, &c);
    return {c, s};
}

// Per-walker constants of the mode model (the "fitting constants" the paper
// computes on the host; here they are derived on the device).
struct Source {
    double M;        // total mass [s]
    double eta, dlt;  // symmetric mass ratio, (1 - q) / (1 + q)
    double chis, chia, chieff;
    double dist;     // luminosity distance [s]
    double phiref, iota, lam, beta, psi;
    double tc;       // t_coal = t_ref + t0 [s]
    double amp0;     // sqrt(2 eta / 3) pi^(-1/6) M^2 / D
    double al2, al3;  // amplitude correction coefficients
    double ps2, ps3;  // phase series coefficients
    double xrd;      // remnant ringdown frequency in M f
    double phj, c1, c2;  // merger-ringdown continuation: phj + c1 (x - xj) - c2 (1/x - 1/xj)
    double xpk, phpk, dphpk;  // peak of f^2 A_22, the raw phase and slope there
    double k128;     // 1 / (128 eta), the leading phase coefficient
    double m2pi;     // M / (2 pi)
};

// Inspiral phase and its first two x-derivatives at x = M f (t_c = 0 frame).
struct PhaseSet {
    double p, dp, d2p;
};
__device__ inline PhaseSet inspiral_phase(const Source &s, double x) {
    const double v = cbrt(kPi * x);
    const double iv = 1.0 / v;
    const double iv2 = iv * iv, iv3 = iv2 * iv, iv5 = iv3 * iv2;
    const double k = 1.0 / (128.0 * s.eta);
    PhaseSet r;
    r.p = -3.0 * k * (iv5 + s.ps2 * iv3 + s.ps3 * iv2);
    r.dp = k / x * (5.0 * iv5 + 3.0 * s.ps2 * iv3 + 2.0 * s.ps3 * iv2);
    r.d2p = -k / (x * x) * ((40.0 / 3.0) * iv5 + 6.0 * s.ps2 * iv3 + (10.0 / 3.0) * s.ps3 * iv2);
    return r;
}

__device__ inline double raw_phase(const Source &s, double x) {
    if (x <= kXJoin) return inspiral_phase(s, x).p;
    return s.phj + s.c1 * (x - kXJoin) - s.c2 * (1.0 / x - 1.0 / kXJoin);
}

__device__ inline double raw_slope(const Source &s, double x) {
    if (x <= kXJoin) return inspiral_phase(s, x).dp;
    return s.c1 + s.c2 / (x * x);
}

// x d ln(f^2 A_22) / dx, whose zero is the peak of f^2 A_22
__device__ inline double peak_equation(const Source &s, double x) {
    const double v = cbrt(kPi * x);
    const double r = x / s.xrd;
    const double r2 = r * r;
    const double r6 = r2 * r2 * r2;
    return 5.0 / 6.0 + (2.0 / 3.0) * s.al2 * v * v + s.al3 * v * v * v - 6.0 * r6 / (1.0 + r6);
}

// Derive the walker constants except the peak of f^2 A_22; false for a walker outside
// the physical range.
__device__ inline bool make_source_core(const double *th, double t0, Source &s) {
    for (int i = 0; i < kNPar; i++)
        if (!isfinite(th[i])) return false;
    const double mt = th[0], q = th[1], a1 = th[2], a2 = th[3], dl = th[4];
    if (!(mt > 0.0) || !(q > 0.0) || !(q <= 1.0) || !(fabs(a1) <= 0.99) ||
        !(fabs(a2) <= 0.99) || !(dl > 0.0) || !isfinite(t0))
        return false;
    const double opq = 1.0 + q;
    s.M = mt * kMsunS;
    s.eta = q / (opq * opq);
    s.dlt = (1.0 - q) / opq;
    s.chis = 0.5 * (a1 + a2);
    s.chia = 0.5 * (a1 - a2);
    s.chieff = (a1 + q * a2) / opq;
    s.dist = dl * kGpcM / kClight;
    s.phiref = th[5];
    s.iota = th[6];
    s.lam = th[7];
    s.beta = th[8];
    s.psi = th[9];
    s.tc = th[10] + t0;
    const double eta = s.eta;
    s.k128 = 1.0 / (128.0 * eta);
    s.m2pi = s.M / kTwoPi;
    s.amp0 = sqrt(2.0 * eta / 3.0) * pow(kPi, -1.0 / 6.0) * s.M * s.M / s.dist;
    s.al2 = -323.0 / 224.0 + 451.0 / 168.0 * eta;
    s.al3 = (27.0 / 8.0 - 11.0 / 6.0 * eta) * s.chis + 27.0 / 8.0 * s.dlt * s.chia;
    s.ps2 = 3715.0 / 756.0 + 55.0 / 9.0 * eta;
    s.ps3 = (113.0 / 3.0 - 76.0 / 3.0 * eta) * s.chis + 113.0 / 3.0 * s.dlt * s.chia;
    // STANDIN remnant: spin, mass and ringdown frequency
    double af = 2.0 * sqrt(3.0) * eta - 3.871 * eta * eta + 4.028 * eta * eta * eta +
                0.3 * s.chieff;
    af = fmin(0.99, fmax(-0.99, af));
    const double mf = 1.0 - 0.0572 * eta - 0.498 * eta * eta;
    s.xrd = (1.0 - 0.63 * pow(1.0 - af, 0.3)) / (2.0 * kPi * mf);
    // merger-ringdown continuation with matching value, slope and curvature
    const PhaseSet j = inspiral_phase(s, kXJoin);
    s.phj = j.p;
    s.c2 = -0.5 * kXJoin * kXJoin * kXJoin * j.d2p;
    s.c1 = j.dp - s.c2 / (kXJoin * kXJoin);
    return true;
}

// peak of f^2 A_22 (t_coal is reached there, Sec. II): bisection on the sign of its
// log-derivative over [x_RD/4, 2 x_RD]
__device__ inline double find_peak(const Source &s) {
    double lo = 0.25 * s.xrd, hi = 2.0 * s.xrd;
    if (peak_equation(s, lo) <= 0.0) return lo;
    if (peak_equation(s, hi) >= 0.0) return hi;
    for (int it = 0; it < 200 && hi - lo > 1e-14 * hi; it++) {
        const double mid = 0.5 * (lo + hi);
        if (peak_equation(s, mid) > 0.0)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

// align the (2,2) phase at the peak: t_22(f_peak) = t_coal and phi_22(f_peak) = 0
__device__ inline void set_peak(Source &s, double xpk) {
    s.xpk = xpk;
    s.phpk = raw_phase(s, xpk);
    s.dphpk = raw_slope(s, xpk);
}

__device__ inline bool make_source(const double *th, double t0, Source &s) {
    if (!make_source_core(th, t0, s)) return false;
    set_peak(s, find_peak(s));
    return true;
}

// ---------------------------------------------------------------- harmonic modes
// Mode table: index 0..5 for (2,2),(3,3),(4,4),(2,1),(3,2),(4,3).
__host__ __device__ inline int mode_index(int l, int m) {
    if (l == 2 && m == 2) return 0;
    if (l == 3 && m == 3) return 1;
    if (l == 4 && m == 4) return 2;
    if (l == 2 && m == 1) return 3;
    if (l == 3 && m == 2) return 4;
    if (l == 4 && m == 3) return 5;
    return -1;
}

struct Mode {
    int l, m;
};

// mode-mapped (2,2) argument x = 2 M f / m
__device__ inline double mapped_x(const Source &s, const Mode &md, double f) {
    return 2.0 * s.M * f / md.m;
}

// Eq. (6): t_lm(f) = t_coal - (1/2pi) dphi_lm/df = t_22(2 f / m)
__device__ inline double mode_time(const Source &s, const Mode &md, double f) {
    const double x = mapped_x(s, md, f);
    return s.tc - s.M / kTwoPi * (raw_slope(s, x) - s.dphpk);
}

__device__ inline double amp_ratio(const Source &s, const Mode &md, double v) {
    double r = 1.0;
    const int id = mode_index(md.l, md.m);
    if (id == 1) r = 0.75 * sqrt(15.0 / 14.0) * s.dlt * v;
    if (id == 2) r = 8.0 / 9.0 * sqrt(5.0 / 7.0) * (1.0 - 3.0 * s.eta) * v * v;
    if (id == 3) r = sqrt(2.0) / 3.0 * s.dlt * v;
    if (id == 4) r = 1.0 / 3.0 * sqrt(5.0 / 7.0) * (1.0 - 3.0 * s.eta) * v * v;
    if (id == 5) r = 9.0 / (4.0 * sqrt(70.0)) * s.dlt * (1.0 - 2.0 * s.eta) * v * v * v;
    // sqrt(2 / m) for m = 1..4
    const double sq = md.m == 1   ? 1.4142135623730951
                      : md.m == 2 ? 1.0
                      : md.m == 3 ? 0.816496580927726
                                  : 0.7071067811865476;
    return r * sq;
}

__device__ inline double phase_offset(const Mode &md) {
    switch (mode_index(md.l, md.m)) {
        case 1: return -0.5 * kPi;
        case 2: return kPi;
        case 3: return 0.5 * kPi;
        case 5: return -0.5 * kPi;
        default: return 0.0;
    }
}

// Eq. (5): A_lm(f) of the stand-in mode model
__device__ inline double mode_amp(const Source &s, const Mode &md, double f) {
    const double x = mapped_x(s, md, f);
    const double v = cbrt(kPi * x);
    const double r = x / s.xrd;
    const double r2 = r * r;
    const double a22 = s.amp0 * pow(x, -7.0 / 6.0) * exp(s.al2 * v * v + s.al3 * v * v * v) /
                       (1.0 + r2 * r2 * r2);
    return amp_ratio(s, md, v) * a22;
}

// Eq. (5): phi_lm(f) = (m/2) phi_22(2 f / m) + const, phi_22 aligned at the peak
__device__ inline double mode_phase(const Source &s, const Mode &md, double f) {
    const double x = mapped_x(s, md, f);
    const double p22 = raw_phase(s, x) - s.phpk - s.dphpk * (x - s.xpk);
    return 0.5 * md.m * p22 + phase_offset(md);
}

// A_lm(f), phi_lm(f) and t_lm(f) together (Eqs. (5), (6)), sharing one cube root:
// x^(-7/6) = 1 / (x sqrt(x^(1/3))) with x^(1/3) = v / pi^(1/3)
__device__ inline void mode_all(const Source &s, const Mode &md, double f, double &amp,
                                double &phase, double &time) {
    const double x = mapped_x(s, md, f);
    const double v = cbrt(kPi * x);
    const double ix = 1.0 / x;
    double p, dp;
    if (x <= kXJoin) {
        const double iv = 1.0 / v;
        const double iv2 = iv * iv, iv3 = iv2 * iv, iv5 = iv3 * iv2;
        const double k = s.k128;
        p = -3.0 * k * (iv5 + s.ps2 * iv3 + s.ps3 * iv2);
        dp = k * ix * (5.0 * iv5 + 3.0 * s.ps2 * iv3 + 2.0 * s.ps3 * iv2);
    } else {
        p = s.phj + s.c1 * (x - kXJoin) - s.c2 * (ix - 1.0 / kXJoin);
        dp = s.c1 + s.c2 * ix * ix;
    }
    time = s.tc - s.m2pi * (dp - s.dphpk);
    phase = 0.5 * md.m * (p - s.phpk - s.dphpk * (x - s.xpk)) + phase_offset(md);
    const double r = x / s.xrd;
    const double r2 = r * r;
    const double x16 = sqrt(v * 0.68278406325529568);  // x^(1/6); 0.6827... = pi^(-1/3)
    const double a22 = s.amp0 * ix * exp(s.al2 * v * v + s.al3 * v * v * v) /
                       (x16 * (1.0 + r2 * r2 * r2));
    amp = amp_ratio(s, md, v) * a22;
}

// -2Y_lm(iota, phi) for l = 2..4 in closed form; (l, m) with |m| from the mode table
__device__ inline cplx ylm_m2(int l, int m, double th, double ph) {
    const double c = cos(0.5 * th), s = sin(0.5 * th), ct = cos(th);
    const double c2 = c * c, s2 = s * s;
    double v = 0.0;
    if (l == 2) {
        if (m == 2) v = sqrt(5.0 / (4.0 * kPi)) * c2 * c2;
        if (m == -2) v = sqrt(5.0 / (4.0 * kPi)) * s2 * s2;
        if (m == 1) v = sqrt(5.0 / kPi) * c2 * c * s;
        if (m == -1) v = sqrt(5.0 / kPi) * s2 * s * c;
    } else if (l == 3) {
        if (m == 3) v = -sqrt(21.0 / (2.0 * kPi)) * c2 * c2 * c * s;
        if (m == -3) v = sqrt(21.0 / (2.0 * kPi)) * s2 * s2 * s * c;
        if (m == 2) v = 0.5 * sqrt(7.0 / kPi) * c2 * c2 * (3.0 * ct - 2.0);
        if (m == -2) v = 0.5 * sqrt(7.0 / kPi) * s2 * s2 * (3.0 * ct + 2.0);
    } else if (l == 4) {
        if (m == 4) v = 3.0 * sqrt(7.0 / kPi) * c2 * c2 * c2 * s2;
        if (m == -4) v = 3.0 * sqrt(7.0 / kPi) * s2 * s2 * s2 * c2;
        if (m == 3) v = -3.0 * sqrt(7.0 / (2.0 * kPi)) * c2 * c2 * c * s * (2.0 * ct - 1.0);
        if (m == -3) v = 3.0 * sqrt(7.0 / (2.0 * kPi)) * s2 * s2 * s * c * (2.0 * ct + 1.0);
    }
    return {v * cos(m * ph), v * sin(m * ph)};
}

// Polarisation weights of the positive-frequency content of mode (l, m):
// h+ = Kp h_lm and hx = Kc h_lm, from h = h+ - i hx = sum h_lm Y_lm and the
// aligned-spin symmetry h_{l,-m}(f) = (-1)^l h*_lm(-f).
__device__ inline void pol_weights(const Source &s, const Mode &md, cplx &kp, cplx &kc) {
    const cplx yp = ylm_m2(md.l, md.m, s.iota, s.phiref);
    const cplx ym = ylm_m2(md.l, -md.m, s.iota, s.phiref);
    const double sg = (md.l & 1) ? -1.0 : 1.0;
    const cplx ypc = {sg * yp.re, -sg * yp.im};  // (-1)^l conj(Y_lm)
    kp = {0.5 * (ym.re + ypc.re), 0.5 * (ym.im + ypc.im)};
    const cplx d = {ym.re - ypc.re, ym.im - ypc.im};
    kc = {-0.5 * d.im, 0.5 * d.re};  // (i/2) d
}

// ---------------------------------------------------------------- orbit and response
struct Frame {
    double k[3];       // propagation direction
    double ep[3][3];   // plus tensor (psi applied)
    double ec[3][3];   // cross tensor (psi applied)
};

__device__ inline void make_frame(const Source &s, Frame &fr) {
    double sl, cl, sb, cb, s2p, c2p;
    sincos(s.lam, &sl, &cl);
    sincos(s.beta, &sb, &cb);
    sincos(2.0 * s.psi, &s2p, &c2p);
    const double u[3] = {sl, -cl, 0.0};
    const double w[3] = {-sb * cl, -sb * sl, cb};
    fr.k[0] = -cb * cl;
    fr.k[1] = -cb * sl;
    fr.k[2] = -sb;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            const double e_p = u[a] * u[b] - w[a] * w[b];
            const double e_c = u[a] * w[b] + w[a] * u[b];
            fr.ep[a][b] = c2p * e_p + s2p * e_c;
            fr.ec[a][b] = -s2p * e_p + c2p * e_c;
        }
}

// constellation centre p0 and spacecraft offsets q[i] (seconds) at time t; the angles
// 2 alpha - b_i and alpha - b_i come from one sincos of alpha by angle addition
__device__ inline void constellation(double t, double p0[3], double q[3][3]) {
    const double R = kAuM / kClight, L = kArmM / kClight;
    const double al = kTwoPi * t / kYearS;
    double sa, ca;
    sincos(al, &sa, &ca);
    p0[0] = R * ca;
    p0[1] = R * sa;
    p0[2] = 0.0;
    const double s2a = 2.0 * sa * ca, c2a = ca * ca - sa * sa;
    const double pre = L / (4.0 * sqrt(3.0));
    const double cb[3] = {1.0, -0.5, -0.5};
    const double sbv[3] = {0.0, 0.8660254037844386, -0.8660254037844386};
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const double c1 = c2a * cb[i] + s2a * sbv[i];  // cos(2 al - b)
        const double s1 = s2a * cb[i] - c2a * sbv[i];  // sin(2 al - b)
        const double c2 = ca * cb[i] + sa * sbv[i];    // cos(al - b)
        q[i][0] = pre * (c1 - 3.0 * cb[i]);
        q[i][1] = pre * (s1 - 3.0 * sbv[i]);
        q[i][2] = -2.0 * sqrt(3.0) * pre * c2;
    }
}

// SSB -> constellation-centre delay phase -2 pi f k.p0(t)
__device__ inline double delay_phase(const Frame &fr, double f, double t) {
    double p0[3], q[3][3];
    constellation(t, p0, q);
    return -kTwoPi * f * (fr.k[0] * p0[0] + fr.k[1] * p0[1] + fr.k[2] * p0[2]);
}

// TDI A, E, T transfer of one mode at (f, t), Eqs. (7)-(10).  The two directions of an
// arm share n n^T (so the polarisation factor) and the propagation phase; only the
// sinc argument differs.  The constellation of constellation() is rigid: every arm
// q_c - q_a has length L exactly (to rounding), so the unit vector is (q_c - q_a) / L;
// the two sinc quotients of an arm share one division.
//
// Six sincos instead of eleven, by angle addition (every identity exact in real
// arithmetic):
//  * x = pi f L: sincos(x) gives the delay operator D = e^{-2ix} and the common factor
//    e^{-ix} of the arms' propagation phases e^{-i pi f (L + k.(q_a + q_c))};
//  * the sinc arguments x (1 -+ k.n) take sin(x) and sincos(x k.n): sin(x (1 -+ k.n)) =
//    sin x cos(x k.n) -+ cos x sin(x k.n), used where 1 -+ k.n >= 1e-3 (there the
//    identity loses at most 1e-13 relative); closer to an arm the direct sine is taken;
//  * the arms (0,1), (0,2), (1,2) have n_02 = n_01 + n_12, so the middle arm's x k.n
//    and its sincos come from the other two; and q_0 + q_1 + q_2 = 0 gives
//    k.(q_0 + q_2) = -k.(q_0 + q_1) - k.(q_1 + q_2), so its propagation phase is the
//    conjugate product of the other two.
__device__ inline double link_sin(double a, double sx, double cx, double sy, double cy,
                                  double sgn, double gap) {
    return gap >= 1e-3 ? sx * cy + sgn * cx * sy : sin(a);
}

__device__ inline void tdi_transfer(const Frame &fr, cplx kp, cplx kc, double f, double t,
                                    cplx out[3], double *delay) {
    double p0[3], q[3][3];
    constellation(t, p0, q);
    if (delay) *delay = -kTwoPi * f * (fr.k[0] * p0[0] + fr.k[1] * p0[1] + fr.k[2] * p0[2]);
    const double L = kArmM / kClight;
    const double pfl = kPi * f * L;
    double sp, cp;
    sincos(pfl, &sp, &cp);
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    double kn[3], kq[3];
    cplx F[3];
#pragma unroll
    for (int e = 0; e < 3; e++) {
        const int a = pa[e], c = pb[e];
        double n[3];
        const double inv = 1.0 / L;
#pragma unroll
        for (int i = 0; i < 3; i++) n[i] = q[c][i] - q[a][i];
        double kne = 0.0, kqe = 0.0, xp = 0.0, xc = 0.0;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            n[i] *= inv;
            kne += fr.k[i] * n[i];
            kqe += fr.k[i] * (q[a][i] + q[c][i]);
        }
#pragma unroll
        for (int i = 0; i < 3; i++) {
            double tp = 0.0, tcx = 0.0;
#pragma unroll
            for (int j = 0; j < 3; j++) {
                tp += fr.ep[i][j] * n[j];
                tcx += fr.ec[i][j] * n[j];
            }
            xp += n[i] * tp;
            xc += n[i] * tcx;
        }
        kn[e] = kne;
        kq[e] = kqe;
        F[e] = {kp.re * xp + kc.re * xc, kp.im * xp + kc.im * xc};
    }
    // the middle arm's k.n from the outer two (n_02 = n_01 + n_12)
    kn[1] = kn[0] + kn[2];
    // e^{-i pi f k.(q_a + q_c)} of the outer arms, the middle one's as their conjugate product
    cplx g[3];
    {
        double s0, c0, s2, c2;
        sincos(kPi * f * kq[0], &s0, &c0);
        sincos(kPi * f * kq[2], &s2, &c2);
        g[0] = {c0, -s0};
        g[2] = {c2, -s2};
        const cplx g02 = cmul(g[0], g[2]);
        g[1] = {g02.re, -g02.im};
    }
    // sincos(x k.n) of the outer arms, the middle one's by angle addition
    double sn[3], cn[3];
    sincos(pfl * kn[0], &sn[0], &cn[0]);
    sincos(pfl * kn[2], &sn[2], &cn[2]);
    sn[1] = sn[0] * cn[2] + cn[0] * sn[2];
    cn[1] = cn[0] * cn[2] - sn[0] * sn[2];
    const cplx ex = {cp, -sp};  // e^{-ix}
    cplx y[3][3];  // y[emitter][receiver]
#pragma unroll
    for (int e = 0; e < 3; e++) {
        const int a = pa[e], c = pb[e];
        const cplx eF = cmul(cmul(ex, g[e]), F[e]);
        const double g1 = 1.0 - kn[e], g2 = 1.0 + kn[e];
        const double a1 = pfl * g1, a2 = pfl * g2;  // a -> c and c -> a
        double s1, s2;
        const double a12 = a1 * a2;
        if (a12 != 0.0) {
            const double r = 1.0 / a12;
            s1 = link_sin(a1, sp, cp, sn[e], cn[e], -1.0, g1) * (a2 * r);
            s2 = link_sin(a2, sp, cp, sn[e], cn[e], 1.0, g2) * (a1 * r);
        } else {
            s1 = (a1 == 0.0) ? 1.0 : sin(a1) / a1;
            s2 = (a2 == 0.0) ? 1.0 : sin(a2) / a2;
        }
        // -i pfl sinc e F
        y[a][c] = {pfl * s1 * eF.im, -pfl * s1 * eF.re};
        y[c][a] = {pfl * s2 * eF.im, -pfl * s2 * eF.re};
    }
    const cplx D = {cp * cp - sp * sp, -2.0 * sp * cp};  // e^{-2ix}
    const cplx D2 = cmul(D, D);
    const cplx fac = {1.0 - D2.re, -D2.im};
    const cplx X = cmul(fac, csub(cadd(y[2][0], cmul(D, y[0][2])), cadd(y[1][0], cmul(D, y[0][1]))));
    const cplx Y = cmul(fac, csub(cadd(y[0][1], cmul(D, y[1][0])), cadd(y[2][1], cmul(D, y[1][2]))));
    const cplx Z = cmul(fac, csub(cadd(y[1][2], cmul(D, y[2][1])), cadd(y[0][2], cmul(D, y[2][0]))));
    const double r2 = 1.0 / sqrt(2.0), r6 = 1.0 / sqrt(6.0), r3 = 1.0 / sqrt(3.0);
    out[0] = cscale(csub(Z, X), r2);
    out[1] = cscale(cadd(csub(X, cscale(Y, 2.0)), Z), r6);
    out[2] = cscale(cadd(cadd(X, Y), Z), r3);
}

// ---------------------------------------------------------------- split precision
// The split-precision knot stage evaluates everything in FP64 like the FP64 path and
// stores the amplitude (times 2^64, far from the FP32 underflow) and the transfer as FP32;
// only the phase series stays FP64.  (Evaluating A and T in FP32 at the knots was tried:
// errors at a knot are common to the whole segment, so they average far less than the
// per-bin FP32 errors of the dense stage, and |d lnL| at SNR 1000 grew about tenfold.)
constexpr double kAmpScale64 = 18446744073709551616.0;  // 2^64

}  // namespace lisa
