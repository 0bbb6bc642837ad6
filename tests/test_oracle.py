"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
limits, finite differences, library routines (scipy's not-a-knot CubicSpline, the
"Scipy"-based spline named in Sec. II.A), numbers printed in the paper, invariants
of Eq. (2) and statistics of Eq. (12).
"""
import math
import os

import numpy as np
import pytest

import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
L_S = 2.5e9 / 299792458.0
R_S = 1.495978707e11 / 299792458.0
MTSUN = 4.925490947641267e-06


def theta_c1(orc):
    th = np.array(W.THETA_C1_Z, dtype=float)
    th[4] = orc.dl_gpc(th[4])
    return th


# ----------------------------------------------------------------------------- spline

@pytest.mark.parametrize("K", [4, 5, 7, 64, 1024])
def test_spline_exact_on_cubics(orc, K):
    rng = np.random.default_rng(K)
    x = np.sort(rng.uniform(1e-4, 1e-1, K)) if K < 64 else np.geomspace(1e-5, 1e-1, K)
    c = rng.standard_normal(4)
    poly = lambda t: c[0] + c[1] * (t / 0.05) + c[2] * (t / 0.05) ** 2 + c[3] * (t / 0.05) ** 3
    coef = orc.spline(x, poly(x))
    f = np.concatenate([x, rng.uniform(x[0], x[-1], 500)])
    err = np.max(np.abs(orc.spline_eval(x, coef, f) - poly(f))) / np.max(np.abs(poly(f)))
    assert err < 1e-11


@pytest.mark.parametrize("K", [4, 6, 33, 256])
def test_spline_matches_scipy_not_a_knot(orc, K):
    from scipy.interpolate import CubicSpline

    rng = np.random.default_rng(100 + K)
    x = np.cumsum(rng.uniform(0.5, 2.0, K)) * 1e-3
    y = rng.standard_normal(K) * 1e3
    coef = orc.spline(x, y)
    ref = CubicSpline(x, y, bc_type="not-a-knot")
    f = np.concatenate([x, rng.uniform(x[0], x[-1], 2000)])
    scale = np.max(np.abs(y))
    assert np.max(np.abs(orc.spline_eval(x, coef, f) - ref(f))) / scale < 1e-11
    # the stored per-segment coefficients are the polynomial ones
    assert np.allclose(coef[:, 3], ref.c[0], rtol=1e-9, atol=1e-9 * np.max(np.abs(ref.c[0])))


def test_spline_segment_rule_on_uneven_knots(orc):
    """Every segment is used for its own interval, including the last one, when the
    knots are far from log-spaced (the log-spaced first guess is then wrong)."""
    from scipy.interpolate import CubicSpline

    K = 40
    for x in (1e-3 + np.geomspace(1e-7, 1e-1, K),          # clustered at the lower end
              np.sort(1e-1 - np.geomspace(1e-5, 9e-2, K))):  # clustered at the upper end
        _check_all_segments(orc, x, CubicSpline)


def _check_all_segments(orc, x, CubicSpline):
    K = x.size
    rng = np.random.default_rng(3)
    y = rng.standard_normal(K)
    coef = orc.spline(x, y)
    mids = 0.5 * (x[1:] + x[:-1])
    f = np.concatenate([mids, x])
    ref = CubicSpline(x, y, bc_type="not-a-knot")(f)
    assert np.max(np.abs(orc.spline_eval(x, coef, f) - ref)) < 1e-10


# ----------------------------------------------------------------------------- harmonics

def _ylm_table(l, m, th, ph):
    """-2Y_lm closed forms (l = 2..4 entries used by PhenomHM), written in cos/sin."""
    c, s = math.cos(th / 2), math.sin(th / 2)
    ct = math.cos(th)
    tab = {
        (2, 2): math.sqrt(5 / (64 * math.pi)) * (1 + ct) ** 2,
        (2, 1): math.sqrt(5 / (16 * math.pi)) * math.sin(th) * (1 + ct),
        (2, 0): math.sqrt(15 / (32 * math.pi)) * math.sin(th) ** 2,
        (2, -1): math.sqrt(5 / (16 * math.pi)) * math.sin(th) * (1 - ct),
        (2, -2): math.sqrt(5 / (64 * math.pi)) * (1 - ct) ** 2,
        (3, 3): -math.sqrt(21 / (2 * math.pi)) * c ** 5 * s,
        (3, 2): math.sqrt(7 / math.pi) * c ** 4 * (3 * ct - 2) / 2,
        (3, -2): math.sqrt(7 / (4 * math.pi)) * (2 + 3 * ct) * s ** 4,
        (3, -3): math.sqrt(21 / (2 * math.pi)) * c * s ** 5,
        (4, 4): 3 * math.sqrt(7 / math.pi) * c ** 6 * s ** 2,
        (4, 3): -3 * math.sqrt(7 / (2 * math.pi)) * c ** 5 * (2 * ct - 1) * s,
        (4, -3): 3 * math.sqrt(7 / (2 * math.pi)) * c * (1 + 2 * ct) * s ** 5,
        (4, -4): 3 * math.sqrt(7 / math.pi) * c ** 2 * s ** 6,
        (2, -1): math.sqrt(5 / (16 * math.pi)) * math.sin(th) * (1 - ct),
    }
    return tab[(l, m)] * complex(math.cos(m * ph), math.sin(m * ph))


def test_sylm_closed_forms(orc):
    rng = np.random.default_rng(5)
    keys = [(2, 2), (2, 1), (2, 0), (2, -1), (2, -2), (3, 3), (3, 2), (3, -2), (3, -3),
            (4, 4), (4, 3), (4, -3), (4, -4)]
    for _ in range(20):
        th, ph = rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi)
        for l, m in keys:
            assert abs(orc.sylm(-2, l, m, th, ph) - _ylm_table(l, m, th, ph)) < 1e-13


def test_sylm_orthonormal(orc):
    x, wx = np.polynomial.legendre.leggauss(40)
    nphi = 32
    phis = 2 * math.pi * np.arange(nphi) / nphi
    lms = [(l, m) for l in (2, 3, 4) for m in range(-l, l + 1)]
    Y = np.array([[[orc.sylm(-2, l, m, math.acos(xx), p) for p in phis] for xx in x]
                  for (l, m) in lms])
    G = np.einsum("aij,bij,i->ab", Y, Y.conj(), wx) * (2 * math.pi / nphi)
    assert np.max(np.abs(G - np.eye(len(lms)))) < 1e-12


# ----------------------------------------------------------------------------- modes

def test_mode_symmetry_reduced_form(orc):
    """h_{l,-m}(f) = (-1)^l h*_{lm}(-f): the reduced m>0 polarisations equal the ones
    built from explicit +m and -m harmonics and negative-frequency content."""
    th = W.theta_table2(1)
    th[6], th[5] = 0.7, 1.3
    f = np.geomspace(2e-4, 2e-2, 17)
    for l, m in W.MODES6:
        a, p, _, _ = orc.mode_eval(th, 0.0, l, m, f)
        h_neg_m = a * np.exp(1j * p)                  # content at f > 0: the (l,-m) mode
        h_pos_m_at_minus_f = (-1) ** l * np.conj(h_neg_m)  # the (l,m) mode at -f
        Yp = _ylm_table(l, m, th[6], th[5])
        Ym = _ylm_table(l, -m, th[6], th[5])
        hf = h_neg_m * Ym                              # h = h+ - i hx at +f
        hmf = h_pos_m_at_minus_f * Yp                  # h at -f
        hp_ref = 0.5 * (hf + np.conj(hmf))
        hc_ref = 0.5j * (hf - np.conj(hmf))
        hp, hc = orc.polarizations(th, 0.0, l, m, f)
        scale = np.max(np.abs(hp_ref)) + np.max(np.abs(hc_ref))
        assert np.max(np.abs(hp - hp_ref)) / scale < 1e-12
        assert np.max(np.abs(hc - hc_ref)) / scale < 1e-12


def test_face_on_22_circular(orc):
    th = W.theta_table2(1)
    th[6] = 0.0
    f = np.geomspace(1e-4, 1e-2, 11)
    hp, hc = orc.polarizations(th, 0.0, 2, 2, f)
    assert np.allclose(np.abs(hp), np.abs(hc), rtol=1e-13)
    assert np.allclose(hc, -1j * hp, rtol=1e-13)


def test_odd_m_modes_vanish_for_equal_mass(orc):
    th = W.theta_table2(1)
    th[1] = 1.0
    f = np.geomspace(1e-4, 1e-2, 5)
    for l, m in ((3, 3), (2, 1), (4, 3)):
        a, _, _, _ = orc.mode_eval(th, 0.0, l, m, f)
        assert np.all(a == 0.0)


def test_dphase_matches_finite_difference(orc):
    rng = np.random.default_rng(7)
    for _ in range(6):
        th = W.theta_table2(1)
        th[0] = 10 ** rng.uniform(4, 8)
        th[1] = rng.uniform(0.05, 1)
        th[2:4] = rng.uniform(-0.99, 0.99, 2)
        fp, fc = orc.peak_and_cut(th)
        for l, m in W.MODES6:
            for frac in (0.05, 0.5, 1.3, 3.0):   # inspiral, join region, merger-ringdown
                f = frac * fp * m / 2
                if abs(2 * f / m * th[0] * MTSUN - 0.018) < 1e-3:
                    continue
                hstep = 1e-5 * f
                _, p, dp, _ = orc.mode_eval(th, 0.0, l, m, np.array([f - hstep, f, f + hstep]))
                fd = (p[2] - p[0]) / (2 * hstep)
                assert abs(fd - dp[1]) <= 1e-6 * abs(dp[1]) + 1e-6 * np.max(np.abs(p)) / hstep * 1e-9


def test_tcoal_at_peak_of_f2A(orc):
    th = W.theta_table2(1)
    t0 = W.T0_YEAR
    fp, _ = orc.peak_and_cut(th)
    f = fp * np.array([0.99, 1.0, 1.01])
    a, _, _, t = orc.mode_eval(th, t0, 2, 2, f)
    assert abs(t[1] - (th[10] + t0)) < 1e-6
    g = f ** 2 * a
    assert g[1] > g[0] and g[1] > g[2]


def test_chirp_time_leading_order(orc):
    """t_coal - t(f) -> (5 M / 256 eta) (pi M f)^(-8/3) as v -> 0 (Eq. (6), TaylorF2)."""
    th = W.theta_table2(1)
    M = th[0] * MTSUN
    eta = th[1] / (1 + th[1]) ** 2
    fp, _ = orc.peak_and_cut(th)
    for x in (1e-7, 1e-8):
        f = np.array([x / M])
        _, _, _, t = orc.mode_eval(th, 0.0, 2, 2, f)
        # the aligned phase adds a constant time shift set at the peak
        _, _, _, tp = orc.mode_eval(th, 0.0, 2, 2, np.array([fp]))
        tau = 5 * M / (256 * eta) * (math.pi * x) ** (-8 / 3)
        v = (math.pi * x) ** (1 / 3)
        assert abs((tp[0] - t[0]) / tau - 1) < 10 * v ** 2


def test_mode_time_mapping_and_band_edges(orc):
    th = W.theta_table2(1)
    g = W.GRID_C2
    t0 = W.T0_YEAR
    f = np.geomspace(1e-4, 1e-2, 9)
    _, _, _, t22 = orc.mode_eval(th, t0, 2, 2, f)
    for l, m in W.MODES6:
        _, _, _, tlm = orc.mode_eval(th, t0, l, m, f * m / 2)
        assert np.allclose(tlm, t22, rtol=0, atol=1e-6)
    b22 = orc.band(th, t0, 2, 2, g.f0, g.df, g.n_bins)
    for l, m in W.MODES6:
        b = orc.band(th, t0, l, m, g.f0, g.df, g.n_bins)
        assert b is not None
        flo, fhi, jlo, jhi = b
        if b22[0] > g.f0 and flo > g.f0:
            assert abs(flo - 0.5 * m * b22[0]) < 1e-12 * flo
        _, _, _, tlo = orc.mode_eval(th, t0, l, m, np.array([flo]))
        assert abs(tlo[0]) < 1e-3 or flo == g.f0
        fj = g.f0 + g.df * np.array([jlo - 1, jlo, jhi, jhi + 1], dtype=float)
        assert fj[1] >= flo - 1e-9 * g.df and fj[0] < flo
        assert fj[2] <= fhi + 1e-9 * g.df and (jhi == g.n_bins - 1 or fj[3] > fhi)


# ----------------------------------------------------------------------------- orbit, response

def test_orbit_rigid_equal_arm():
    import oracle as orc

    for t in np.linspace(0, 3.15576e7, 13):
        p0, q = orc.orbit(t)
        assert abs(np.linalg.norm(p0) - R_S) < 1e-12 * R_S
        assert np.allclose(q.sum(axis=0), 0.0, atol=1e-13)
        for i in range(3):
            assert abs(np.linalg.norm(q[i]) - L_S / math.sqrt(3)) < 1e-13 * L_S
            for j in range(i):
                assert abs(np.linalg.norm(q[i] - q[j]) - L_S) < 1e-13 * L_S
        nrm = np.cross(q[1] - q[0], q[2] - q[0])
        nrm /= np.linalg.norm(nrm)
        assert abs(abs(nrm[2]) - 0.5) < 1e-12   # plane inclined by 60 degrees


def _pol_tensors(lam, beta, psi):
    u = np.array([math.sin(lam), -math.cos(lam), 0.0])
    v = np.array([-math.sin(beta) * math.cos(lam), -math.sin(beta) * math.sin(lam), math.cos(beta)])
    ep, ec = np.outer(u, u) - np.outer(v, v), np.outer(u, v) + np.outer(v, u)
    return (math.cos(2 * psi) * ep + math.sin(2 * psi) * ec,
            -math.sin(2 * psi) * ep + math.cos(2 * psi) * ec)


def test_response_long_wavelength_limit(orc):
    """As f L -> 0 the transfer tends to X = 8 pi^2 f^2 L^2 (F(n_13) - F(n_12)) with
    F(n) = K+ n.E+.n + Kx n.Ex.n, and A, E, T of Eqs. (8)-(10) of X, Y, Z."""
    th = W.theta_table2(1)
    f, t = 1e-6, 1.1e7
    for l, m in ((2, 2), (3, 3)):
        T = orc.transfer(th, l, m, np.array([f]), np.array([t]))[:, 0]
        _, q = orc.orbit(t)
        Ep, Ec = _pol_tensors(th[7], th[8], th[9])
        Yp = _ylm_table(l, m, th[6], th[5])
        Ym = _ylm_table(l, -m, th[6], th[5])
        Kp = 0.5 * (Ym + (-1) ** l * np.conj(Yp))
        Kc = 0.5j * (Ym - (-1) ** l * np.conj(Yp))

        def F(a, b):
            n = (q[b] - q[a]) / np.linalg.norm(q[b] - q[a])
            return Kp * (n @ Ep @ n) + Kc * (n @ Ec @ n)

        pre = 8 * math.pi ** 2 * f ** 2 * L_S ** 2
        X = pre * (F(0, 2) - F(0, 1))
        Y = pre * (F(1, 0) - F(1, 2))
        Z = pre * (F(2, 1) - F(2, 0))
        A = (Z - X) / math.sqrt(2)
        E = (X - 2 * Y + Z) / math.sqrt(6)
        fl = math.pi * f * L_S
        assert abs(T[0] - A) < 1e-3 * abs(A) + 10 * fl * abs(pre)
        assert abs(T[1] - E) < 1e-3 * abs(E) + 10 * fl * abs(pre)
        assert abs(T[2]) < 10 * fl * max(abs(T[0]), abs(T[1]))   # T suppressed at low f


def test_response_polarisation_symmetry(orc):
    th = W.theta_table2(1)
    f = np.geomspace(1e-4, 5e-2, 7)
    t = np.linspace(1e6, 3e7, 7)
    T0 = orc.transfer(th, 2, 2, f, t)
    th2 = th.copy()
    th2[9] += math.pi / 2
    th3 = th.copy()
    th3[9] += math.pi
    assert np.allclose(orc.transfer(th2, 2, 2, f, t), -T0, rtol=1e-12, atol=1e-14 * np.abs(T0).max())
    assert np.allclose(orc.transfer(th3, 2, 2, f, t), T0, rtol=1e-12, atol=1e-14 * np.abs(T0).max())
    # the transfer is extrinsic: independent of mass, spins and distance
    th4 = th.copy()
    th4[0], th4[1], th4[2], th4[4] = 3e5, 0.7, 0.5, 3.0
    assert np.array_equal(orc.transfer(th4, 2, 2, f, t), T0)


def test_delay_phase_is_the_roemer_delay(orc):
    """The SSB -> constellation-centre phase equals -2 pi f times the arrival delay
    t_L - t of the wave at the centre.  Two independent sources of that delay: the
    sampler oracle's frame conversion (its own orbit and sky vectors), and k.p0 from
    the orbit with the propagation direction k = -(cos b cos l, cos b sin l, sin b)."""
    rng = np.random.default_rng(11)
    for _ in range(12):
        th = W.theta_table2(1).copy()
        th[7] = rng.uniform(0.0, 2 * math.pi)
        th[8] = math.asin(rng.uniform(-1.0, 1.0))
        th[9] = rng.uniform(0.0, math.pi)
        t = rng.uniform(0.0, 3.15576e7)
        f = 10 ** rng.uniform(-5.0, -1.0)
        tL = orc.ssb_to_lisa(t, th[7], th[8], th[9])[0]
        ph = orc.delay_phase(th, f, t)
        assert abs(ph - (-2 * math.pi * f * (tL - t))) <= 1e-9 * abs(2 * math.pi * f * R_S)
        p0, _ = orc.orbit(t)
        k = -np.array([math.cos(th[8]) * math.cos(th[7]), math.cos(th[8]) * math.sin(th[7]),
                       math.sin(th[8])])
        assert abs(ph + 2 * math.pi * f * (k @ p0)) <= 1e-12 * abs(2 * math.pi * f * R_S)
    # at 0.1 Hz a source in the ecliptic plane along the Earth-Sun line has |phase| ~ 2 pi f AU
    th = W.theta_table2(1).copy()
    th[7], th[8] = 0.0, 0.0
    assert abs(abs(orc.delay_phase(th, 0.1, 0.0)) - 2 * math.pi * 0.1 * R_S) < 1e-9 * R_S


def _link_by_quadrature(P, k, f, xs, xr, t_r):
    """Fractional frequency shift of the link s -> r for light received at xr at t_r
    from a plane wave h_ij(t, x) = P_ij exp(2 pi i f (t - k.x)), positions frozen:
    y = -1/2 n.(integral of dh/dt along the light path).n, by 64-point Gauss-Legendre
    (no closed form of the path integral is used)."""
    Lsr = np.linalg.norm(xr - xs)
    n = (xr - xs) / Lsr
    z, wq = np.polynomial.legendre.leggauss(64)
    tau = t_r - 0.5 * Lsr * (1.0 - z)            # emission t_r - L .. reception t_r
    x = xs[None, :] + np.outer(tau - (t_r - Lsr), n)
    dh = 2j * math.pi * f * (n @ P @ n) * np.exp(2j * math.pi * f * (tau - x @ k))
    return -0.5 * 0.5 * Lsr * np.sum(wq * dh)


def _tdi_time_domain(P, k, f, pos, t):
    """First-generation X, Y, Z at time t from explicitly delayed links: the round
    trip a -> b -> a received at a at t is y_{b->a}(t) + y_{a->b}(t - L), and
    X = [0->2->0](t) - [0->1->0](t) - [0->2->0](t - 2L) + [0->1->0](t - 2L), Y and Z
    by cyclic permutation of the spacecraft.  Times are taken relative to t (the wave's
    phase origin there), which keeps the large phase 2 pi f t out of the rounding."""
    L = np.linalg.norm(pos[1] - pos[0])

    def rt(a, b, tt):
        return (_link_by_quadrature(P, k, f, pos[b], pos[a], tt) +
                _link_by_quadrature(P, k, f, pos[a], pos[b], tt - L))

    def mich(a, b, c):
        return rt(a, c, t) - rt(a, b, t) - rt(a, c, t - 2 * L) + rt(a, b, t - 2 * L)

    return mich(0, 1, 2), mich(1, 2, 0), mich(2, 0, 1)


@pytest.mark.parametrize("fL", [0.05, 0.3, 0.83, 1.7])
def test_response_matches_time_domain_tdi_at_finite_fL(orc, fL):
    """Eqs. (7)-(10) at finite f L against a time-domain computation for a frozen
    constellation: a monochromatic plane wave with the mode's polarisation factors,
    each link integrated along the light path, X, Y, Z formed with explicit L delays,
    then A, E, T.  With the spacecraft offsets q relative to the centre this is the
    transfer; with the absolute positions p0 + q it is the transfer times
    exp(i delay phase).  This fixes the sinc argument, the sign of the link exponent,
    the delay operators and the sign of the delay phase at finite f L.  (f L = 1/2,
    1, 3/2, ... are avoided: there 1 - D^2 = 0 and every first-generation channel
    vanishes.)"""
    f = fL / L_S
    rng = np.random.default_rng(int(fL * 1000))
    for l, m in ((2, 2), (3, 3), (2, 1)):
        th = W.theta_table2(1).copy()
        th[5], th[6] = rng.uniform(0, 2 * math.pi), rng.uniform(0.2, 2.9)
        th[7], th[8] = rng.uniform(0, 2 * math.pi), math.asin(rng.uniform(-1, 1))
        th[9] = rng.uniform(0, math.pi)
        t = rng.uniform(0.0, 3.15576e7)
        T = orc.transfer(th, l, m, np.array([f]), np.array([t]))[:, 0]
        p0, q = orc.orbit(t)
        Ep, Ec = _pol_tensors(th[7], th[8], th[9])
        Yp = _ylm_table(l, m, th[6], th[5])
        Ym = _ylm_table(l, -m, th[6], th[5])
        Kp = 0.5 * (Ym + (-1) ** l * np.conj(Yp))
        Kc = 0.5j * (Ym - (-1) ** l * np.conj(Yp))
        P = Kp * Ep + Kc * Ec
        k = -np.array([math.cos(th[8]) * math.cos(th[7]), math.cos(th[8]) * math.sin(th[7]),
                       math.sin(th[8])])
        scale = np.abs(T).max()
        assert scale > 0
        for pos, rot in ((q, 1.0), (p0[None, :] + q, np.exp(1j * orc.delay_phase(th, f, t)))):
            X, Y, Z = _tdi_time_domain(P, k, f, pos, 0.0)
            A = (Z - X) / math.sqrt(2)
            E = (X - 2 * Y + Z) / math.sqrt(6)
            Tc = (X + Y + Z) / math.sqrt(3)
            want = np.array([A, E, Tc])
            assert np.abs(T * rot - want).max() <= 1e-10 * scale, (l, m, fL)


# ----------------------------------------------------------------------------- likelihood

def test_zero_noise_injection_lnL_zero(orc):
    g = W.GRID_C1
    th = theta_c1(orc)
    f = g.freqs()
    S = orc.psd_aet(f)
    d = orc.template(th, W.T0_C1, [(2, 2)], 256, g.f0, g.df, g.n_bins)
    lnL, dh, hh, dd = orc.loglike(th, W.T0_C1, [(2, 2)], 256, g.f0, g.df, d, S, n_threads=1)
    snr2 = orc.inner(d, d, S, g.df)
    assert snr2 > 100.0
    assert abs(lnL[0]) <= 1e-12 * snr2
    assert abs(hh[0] - snr2) <= 1e-12 * snr2 and abs(dh[0] - snr2) <= 1e-12 * snr2
    assert abs(dd - snr2) <= 1e-12 * snr2
    # any other walker is less likely
    th2 = th.copy()
    th2[0] *= 1.001
    lnL2, _, _, _ = orc.loglike(th2, W.T0_C1, [(2, 2)], 256, g.f0, g.df, d, S, n_threads=1)
    assert lnL2[0] < -1e-3


def test_two_algebraic_forms_agree_with_noise(orc):
    g = W.GRID_C1
    th = theta_c1(orc)
    S = orc.psd_aet(g.freqs())
    d = orc.template(th, W.T0_C1, [(2, 2)], 256, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 2))
    th2 = th.copy()
    th2[5] += 0.1
    lnL, _, _, dd = orc.loglike(th2, W.T0_C1, [(2, 2)], 256, g.f0, g.df, d, S, n_threads=1)
    lnL_res = orc.loglike_residual(th2, W.T0_C1, [(2, 2)], 256, g.f0, g.df, d, S)
    assert abs(lnL[0] - lnL_res) <= 1e-12 * dd


def test_hh_scales_as_inverse_distance_squared(orc):
    g = W.GRID_C1
    th = theta_c1(orc)
    S = orc.psd_aet(g.freqs())
    d = np.zeros((3, g.n_bins), complex)
    th2 = th.copy()
    th2[4] *= 2.0
    _, _, hh1, _ = orc.loglike(th, W.T0_C1, [(2, 2)], 256, g.f0, g.df, d, S, n_threads=1)
    _, _, hh2, _ = orc.loglike(th2, W.T0_C1, [(2, 2)], 256, g.f0, g.df, d, S, n_threads=1)
    assert abs(hh2[0] * 4.0 / hh1[0] - 1.0) < 1e-13


def test_spline_template_converges_to_direct(orc):
    """Knots -> spline -> bins approximates direct evaluation with error O(K^-4)."""
    th = W.theta_table2(1)
    th[0] = 1e6
    f0, df, n = 1e-3, 1e-6, 2001
    S = orc.psd_aet(f0 + df * np.arange(n))
    hd = orc.direct(th, W.T0_YEAR, [(2, 2)], f0, df, n)
    norm = orc.inner(hd, hd, S, df)
    errs = []
    for K in (16, 32, 64, 128):
        h = orc.template(th, W.T0_YEAR, [(2, 2)], K, f0, df, n)
        errs.append(math.sqrt(orc.inner(h - hd, h - hd, S, df) / norm))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert errs[-1] < 1e-6
    assert min(orders) > 3.5, (errs, orders)


def test_invalid_walkers_get_minus_inf(orc):
    g = W.GRID_C1
    th = theta_c1(orc)
    S = orc.psd_aet(g.freqs())
    d = np.zeros((3, g.n_bins), complex)
    bad = np.repeat(th[None, :], 6, axis=0)
    bad[0, 1] = 1.5
    bad[1, 2] = 0.995
    bad[2, 0] = -1.0
    bad[3, 4] = 0.0
    bad[4, 6] = np.nan
    lnL, _, _, _ = orc.loglike(bad, W.T0_C1, [(2, 2)], 256, g.f0, g.df, d, S, n_threads=1)
    assert np.all(np.isneginf(lnL[:5])) and np.isfinite(lnL[5])


def test_noise_chi2(orc):
    g = W.GRID_C1
    S = orc.psd_aet(g.freqs())
    n = orc.noise(S, g.df, W.white_noise(g.n_bins, 11))
    nn = orc.inner(n, n, S, g.df)
    per_bin = nn / (3 * g.n_bins)
    assert abs(per_bin - 2.0) < 3 * math.sqrt(4.0 / (3 * g.n_bins))


def test_psd_shape(orc):
    f = np.geomspace(1e-5, 1e-1, 400)
    S = orc.psd_aet(f)
    assert np.all(np.isfinite(S)) and np.all(S > 0)
    assert np.array_equal(S[0], S[1])
    assert np.all(S[2][f < 1e-3] < S[0][f < 1e-3])


def test_distance_redshift_golden(orc):
    rows = [ln.split() for ln in open(os.path.join(GOLD, "distance_redshift.txt"))
            if ln.strip() and not ln.startswith("#")]
    for z, dl, tol, _src in rows:
        z, dl, tol = float(z), float(dl), float(tol)
        got = orc.dl_gpc(z)
        # printed to the digits shown; the stand-in cosmology is also allowed 0.5 %
        assert abs(got - dl) <= max(tol, 0.005 * dl) + 0.0006, (z, got, dl)


def test_binary1_mode_ordering_matches_table3(orc):
    """Sanity shape only (true PhenomHM is not available): the per-mode SNR ordering
    of Binary 1 in Table III."""
    rows = [ln.split() for ln in open(os.path.join(GOLD, "table3_mode_snr.txt"))
            if ln.strip() and not ln.startswith("#")]
    b1 = [float(v) for v in rows[0][2:]]
    g = W.Grid.spanning(1e-5, 1e-1, 1.0 / W.YEAR_S)
    g = W.Grid(g.f0, g.df * 8, g.n_bins // 8)    # coarser grid keeps the test fast
    th = W.theta_table2(1)
    S = orc.psd_aet(g.freqs())
    snr = []
    for md in W.MODES6:
        h = orc.template(th, W.T0_YEAR, [md], 512, g.f0, g.df, g.n_bins)
        snr.append(math.sqrt(orc.inner(h, h, S, g.df)))
    assert np.argsort(snr).tolist() == np.argsort(b1).tolist()
