"""Pins of the oracle's ensemble sampler (Sec. III) against what the mathematics fixes:
published Philox known-answer vectors, the stationary distributions of the stretch move
and of parallel tempering on targets whose moments are known in closed form, the
autocorrelation estimator against an independent FFT computation and the AR(1) closed
form, the default ladder of Sec. III.B, and the LISA-frame conversion against the
geometry of the constellation computed from the orbit itself."""
import math

import numpy as np
import pytest

import workloads as W

D = 11
BOX_LO, BOX_HI = np.full(D, -60.0), np.full(D, 60.0)
MEAN = np.linspace(-1.0, 1.0, D)
SIGMA = np.linspace(0.5, 2.0, D)


def tau_fft(series):
    """Sec. III.C estimator computed independently: FFT autocovariance per walker with
    the 1/(N - t) normalisation, averaged over walkers, Sokal window M >= 5 tau."""
    n, _ = series.shape
    x = series - series.mean(axis=0)
    f = np.fft.rfft(x, 2 * n, axis=0)
    ac = np.fft.irfft(f * np.conj(f), axis=0)[:n] / (n - np.arange(n))[:, None]
    rho = (ac / ac[0]).mean(axis=1)
    tau = 1.0
    for M in range(1, n):
        tau += 2.0 * rho[M]
        if M >= 5.0 * tau:
            break
    return tau, rho


def ar1(n, walkers, phi, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((n, walkers))
    x = np.empty((n, walkers))
    x[0] = e[0] / math.sqrt(1.0 - phi * phi)
    for i in range(1, n):
        x[i] = phi * x[i - 1] + e[i]
    return x


def moment_z(chain, mean, sigma, beta=1.0):
    """z-scores of the sample mean and variance of every coordinate against N(mean,
    sigma^2 / beta), with the effective sample size from the FFT estimator."""
    n, walkers, _ = chain.shape
    flat = chain.reshape(-1, D)
    tau = np.array([tau_fft(chain[:, :, q])[0] for q in range(D)])
    n_eff = n * walkers / tau
    s = sigma / math.sqrt(beta)
    zm = (flat.mean(axis=0) - mean) / (s / np.sqrt(n_eff))
    zv = (flat.var(axis=0) / s ** 2 - 1.0) / np.sqrt(2.0 / n_eff)
    return zm, zv


def start(T, walkers, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    return MEAN + spread * SIGMA * rng.standard_normal((T, walkers, D))


def test_philox_known_answer_vectors(orc):
    """Philox4x32-10 known-answer vectors published with the generator (Salmon et al.
    2011, Random123 distribution)."""
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        assert orc.philox(ctr, key).tolist() == list(want)


def test_default_ladder_is_the_papers():
    """Sec. III.B: ten temperatures, the hottest infinite, the others geometric between
    1 and 2.04807^8."""
    import oracle as orc

    b = orc.default_ladder(10, 2.04807, True)
    assert b[0] == 1.0 and b[9] == 0.0
    T = 1.0 / b[:9]
    assert abs(T[8] - 2.04807 ** 8) <= 1e-9 * T[8]
    assert np.allclose(T[1:] / T[:-1], 2.04807, rtol=1e-13)


def test_autocorr_time_matches_fft_and_ar1_closed_form(orc):
    phi = 0.9
    x = ar1(20000, 16, phi, 0)
    tau, rho = orc.autocorr_time(x, return_rho=True)
    tf, rf = tau_fft(x)
    M = int(5 * tau) + 2
    assert np.max(np.abs(rho[:M] - rf[:M])) <= 1e-12
    assert abs(tau - tf) <= 1e-10 * tf
    # AR(1): tau = (1 + phi) / (1 - phi) = 19; the estimator's error at N = 1000 tau
    assert abs(tau - (1 + phi) / (1 - phi)) <= 0.1 * 19.0
    # white noise: tau = 1
    assert abs(orc.autocorr_time(ar1(20000, 8, 0.0, 1)) - 1.0) <= 0.1


def test_stretch_move_recovers_a_gaussian(orc):
    """One temperature: mean and variance of N(mu, sigma^2) in 11 dimensions."""
    r = orc.sampler_gauss(start(1, 32, 1), [1.0], MEAN, SIGMA, 20000, 11, BOX_LO, BOX_HI, a=2.0)
    zm, zv = moment_z(r.chain[1000:], MEAN, SIGMA)
    assert np.max(np.abs(zm)) < 4.5 and np.max(np.abs(zv)) < 4.5, (zm, zv)
    af = r.acc[0, 0] / r.acc[0, 1]
    assert 0.3 < af < 0.5
    # the paper's scale a = 1.15 accepts more often and still targets the same law
    r = orc.sampler_gauss(start(1, 32, 2), [1.0], MEAN, SIGMA, 20000, 12, BOX_LO, BOX_HI, a=1.15)
    assert r.acc[0, 0] / r.acc[0, 1] > 0.8
    zm, zv = moment_z(r.chain[2000:], MEAN, SIGMA)
    assert np.max(np.abs(zm)) < 5.0 and np.max(np.abs(zv)) < 5.0, (zm, zv)


def test_tempered_chains_sample_the_tempered_target(orc):
    """The coldest chain of a ladder whose coldest beta is 1/4 samples N(mu, 4 sigma^2);
    a wrong swap rule would leak the hotter (8 sigma^2) states into it."""
    r = orc.sampler_gauss(start(2, 32, 3, 2.0), [0.25, 0.125], MEAN, SIGMA, 20000, 13, BOX_LO,
                          BOX_HI, a=2.0)
    zm, zv = moment_z(r.chain[1000:], MEAN, SIGMA, beta=0.25)
    assert np.max(np.abs(zm)) < 4.5 and np.max(np.abs(zv)) < 4.5, (zm, zv)
    rate = r.swaps[0, 0] / r.swaps[0, 1]
    assert 0.1 < rate < 0.5
    assert r.swaps[1, 1] == 0                       # no pair above the hottest
    # a four-rung ladder with beta = 1 at the bottom recovers the target itself
    r = orc.sampler_gauss(start(4, 32, 4), [1.0, 0.5, 0.25, 0.125], MEAN, SIGMA, 20000, 14,
                          BOX_LO, BOX_HI, a=2.0)
    zm, zv = moment_z(r.chain[1000:], MEAN, SIGMA)
    assert np.max(np.abs(zm)) < 4.5 and np.max(np.abs(zv)) < 4.5, (zm, zv)


def test_infinite_temperature_samples_the_prior_box(orc):
    """beta = 0: the stationary law is the uniform prior; without the z^(D-1) factor of
    Eq. (16) the ensemble would contract."""
    lo, hi = np.full(D, -1.0), np.full(D, 3.0)
    rng = np.random.default_rng(5)
    x0 = rng.uniform(lo, hi, size=(1, 32, D))
    r = orc.sampler_gauss(x0, [0.0], MEAN, SIGMA, 20000, 15, lo, hi, a=2.0)
    ch = r.chain[1000:]
    tau = np.array([tau_fft(ch[:, :, q])[0] for q in range(D)])
    n_eff = ch.shape[0] * ch.shape[1] / tau
    flat = ch.reshape(-1, D)
    var_u = (hi - lo) ** 2 / 12.0
    zm = (flat.mean(axis=0) - 1.0) / np.sqrt(var_u / n_eff)
    # variance of the sample variance of a uniform: (mu4 - sigma^4) / n, mu4 = 9/5 sigma^4
    zv = (flat.var(axis=0) - var_u) / np.sqrt(0.8 * var_u ** 2 / n_eff)
    assert np.max(np.abs(zm)) < 4.5 and np.max(np.abs(zv)) < 4.5, (zm, zv)
    assert np.all(flat >= lo) and np.all(flat <= hi)


def test_adaptive_ladder_equalises_swap_rates(orc):
    """Vousden et al. (2016): the ladder moves until adjacent pairs swap equally often;
    the coldest and hottest temperatures stay put."""
    betas = [1.0, 0.9, 0.8, 0.1, 0.05, 0.0]
    x0 = start(6, 32, 6, 3.0)
    fixed = orc.sampler_gauss(x0, betas, MEAN, SIGMA, 4000, 16, BOX_LO, BOX_HI, a=2.0)
    rf = fixed.swaps[:5, 0] / fixed.swaps[:5, 1]
    assert rf.max() > 4 * rf.min()                 # the hand-made ladder is unbalanced
    warm = orc.sampler_gauss(x0, betas, MEAN, SIGMA, 8000, 16, BOX_LO, BOX_HI, a=2.0,
                             adaptive=True, adapt_lag=1000.0, adapt_time=10.0)
    late = orc.sampler_gauss(warm.x, warm.betas, MEAN, SIGMA, 8000, 17, BOX_LO, BOX_HI, a=2.0,
                             step0=8000, adaptive=True, adapt_lag=1000.0, adapt_time=10.0)
    ra = late.swaps[:5, 0] / late.swaps[:5, 1]
    assert ra.max() < 1.6 * ra.min(), ra
    assert late.betas[0] == 1.0 and late.betas[5] == 0.0
    assert np.all(np.diff(late.betas) < 0)


def test_adapt_step_keeps_ends_and_is_neutral_for_equal_rates(orc):
    b = np.array([1.0, 0.5, 0.2, 0.05, 0.0])
    assert np.array_equal(orc.adapt_ladder(b, [0.3, 0.3, 0.3, 0.3, 0.0], 0.1)[:3], b[:3])
    nb = orc.adapt_ladder(b, [0.9, 0.1, 0.3, 0.3, 0.0], 0.5)
    assert nb[0] == 1.0 and nb[4] == 0.0
    # pair 0 accepts more than pair 1: the first gap widens
    assert 1.0 / nb[1] - 1.0 > 1.0 / b[1] - 1.0


def lisa_frame_from_orbit(orc, t):
    """Orthonormal frame in which the spacecraft are at rest, from the orbit alone:
    spacecraft 0 on -x, spacecraft 2 - spacecraft 1 along +y."""
    _, q = orc.orbit(t)
    ex = -q[0] / np.linalg.norm(q[0])
    ey = (q[2] - q[1]) / np.linalg.norm(q[2] - q[1])
    ez = np.cross(ex, ey)
    return np.stack([ex, ey, ez], axis=1)


def sky(lam, beta, psi):
    cl, sl, cb, sb = math.cos(lam), math.sin(lam), math.cos(beta), math.sin(beta)
    n = np.array([cb * cl, cb * sl, sb])
    u = np.array([sl, -cl, 0.0])
    v = np.array([-sb * cl, -sb * sl, cb])
    return n, math.cos(psi) * u + math.sin(psi) * v


def test_lisa_frame_conversion_follows_the_constellation(orc):
    rng = np.random.default_rng(7)
    for _ in range(20):
        tL = rng.uniform(0.0, 3.0 * W.YEAR_S)
        lamL, betL, psiL = rng.uniform(0, 2 * np.pi), math.asin(rng.uniform(-1, 1)), rng.uniform(0, np.pi)
        t, lam, bet, psi = orc.lisa_to_ssb(tL, lamL, betL, psiL)
        Q = lisa_frame_from_orbit(orc, tL)
        nL, pL = sky(lamL, betL, psiL)
        n, p = sky(lam, bet, psi)
        assert np.max(np.abs(n - Q @ nL)) <= 1e-12
        assert abs(abs(p @ (Q @ pL)) - 1.0) <= 1e-12      # same axis (psi is defined mod pi)
        # arrival at the constellation centre: t_L = t + k . p0(t), k = -n
        p0, _ = orc.orbit(t)
        assert abs(tL - (t - n @ p0)) <= 1e-6
        assert abs(tL - t) <= 500.0
        back = orc.ssb_to_lisa(t, lam, bet, psi)
        assert abs(back[0] - tL) <= 1e-6
        assert abs((back[1] - lamL + np.pi) % (2 * np.pi) - np.pi) <= 1e-10
        assert abs(back[2] - betL) <= 1e-10
        assert abs((back[3] - psiL + np.pi / 2) % np.pi - np.pi / 2) <= 1e-10


def test_spacecraft_and_normal_directions_in_the_lisa_frame(orc):
    """A source in the direction of spacecraft 0 sits at beta_L = 0, lambda_L = pi; one
    along the constellation normal at beta_L = pi/2."""
    tL = 0.3 * W.YEAR_S
    _, q = orc.orbit(tL)
    Q = lisa_frame_from_orbit(orc, tL)
    for target, lam_want, bet_want in ((q[0] / np.linalg.norm(q[0]), math.pi, 0.0),
                                       (Q[:, 2], None, math.pi / 2)):
        # find the LISA-frame angles that map onto the target direction
        nL = Q.T @ target
        lamL = math.atan2(nL[1], nL[0]) % (2 * math.pi)
        betL = math.asin(max(-1.0, min(1.0, nL[2])))
        if lam_want is not None:
            assert abs(lamL - lam_want) <= 1e-12
        assert abs(betL - bet_want) <= 1e-7
        _, lam, bet, _ = orc.lisa_to_ssb(tL, lamL, betL, 0.3)
        n, _ = sky(lam, bet, 0.3)
        assert np.max(np.abs(n - target)) <= 1e-7


def test_to_physical_inverts_the_sampling_coordinates(orc):
    x = np.array([math.log(2e6), 0.5, 0.3, -0.2, math.log(25.0), 1.0, 0.3, 2.0, -0.4, 0.7,
                  math.log(3600.0)])
    th = orc.to_physical(x, False, 0.0)
    assert abs(th[0] - 2e6) <= 1e-6 and abs(th[4] - 25.0) <= 1e-12
    assert abs(math.cos(th[6]) - 0.3) <= 1e-15 and abs(math.sin(th[8]) + 0.4) <= 1e-15
    assert abs(th[10] - 3600.0) <= 1e-9 and np.array_equal(th[1:4], x[1:4])
    thL = orc.to_physical(x, True, W.T0_YEAR)
    want = orc.lisa_to_ssb(3600.0 + W.T0_YEAR, 2.0, math.asin(-0.4), 0.7)
    assert np.allclose(thL[7:10], want[1:], atol=1e-14)
    assert abs(thL[10] - (want[0] - W.T0_YEAR)) <= 1e-6


def test_lisa_sampler_state_is_consistent_with_the_likelihood(orc):
    """A few steps on the LISA likelihood: the ln L the sampler carries for each walker
    is the oracle ln L of that walker's physical parameters."""
    g = W.GRID_C1
    S = orc.psd_aet(g.freqs())
    inj = np.array(W.THETA_C1_Z)
    inj[4] = orc.dl_gpc(inj[4])
    inj[10] = 100.0
    d = orc.template(inj, W.T0_C1, [(2, 2)], 64, g.f0, g.df, g.n_bins)
    lo, hi = W.TABLE1_LOWER, W.TABLE1_UPPER
    xc = orc.from_physical(inj)
    rng = np.random.default_rng(8)
    x0 = xc + 1e-4 * rng.standard_normal((2, 8, D))
    r = orc.sampler_lisa(x0, [1.0, 0.5], 3, 21, lo, hi, W.T0_C1, [(2, 2)], 64, g.f0, g.df, d, S,
                         lisa_frame=False)
    th = np.array([orc.to_physical(v, False, W.T0_C1) for v in r.x.reshape(-1, D)])
    ref, _, _, _ = orc.loglike(th, W.T0_C1, [(2, 2)], 64, g.f0, g.df, d, S)
    assert np.allclose(r.lnl.reshape(-1), ref, rtol=0, atol=1e-9)
    assert r.acc[:, 1].tolist() == [24, 24] and r.swaps[0, 1] == 24


def test_partners_come_from_the_other_half(orc):
    """Sec. III.A with the two-half split: with the second half parked at the origin and a
    flat target, every accepted move of a first-half walker is y = z x_k with
    z in [1/a, a], i.e. along the ray from the origin through its old position."""
    rng = np.random.default_rng(9)
    x0 = np.zeros((1, 16, D))
    x0[0, :8] = rng.uniform(1.0, 2.0, size=(8, D))
    a = 2.0
    for seed in range(5):
        r = orc.sampler_gauss(x0, [0.0], MEAN, SIGMA, 1, seed, BOX_LO, BOX_HI, a=a)
        moved = 0
        for k in range(8):
            old, new = x0[0, k], r.x[0, k]
            if np.array_equal(old, new):
                continue
            moved += 1
            z = new / old
            assert np.allclose(z, z[0], rtol=1e-12), "move not along x_k: wrong partner"
            assert 1.0 / a - 1e-12 <= z[0] <= a + 1e-12
        assert moved > 0
