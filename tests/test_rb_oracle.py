"""Pins of the oracle's relative-binning likelihood against what its definition fixes:
exactness at the fiducial and for any template whose ratio to the fiducial is constant
(a distance rescaling), summary data that add up to the dense inner products, and the
second-order convergence of the linear-ratio approximation as the bins shrink."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle_rb as R

MODES = [(2, 2), (3, 3), (4, 4)]


@pytest.fixture(scope="module")
def setup(orc):
    g = W.GRID_C1
    S = orc.psd_aet(g.freqs())
    th = np.array(W.THETA_C1_Z)
    th[4] = orc.dl_gpc(th[4])
    th[10] = 1000.0
    d = orc.direct(th, W.T0_C1, MODES, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 3))
    dd = orc.inner(d, d, S, g.df)
    return g, S, th, d, dd


def dense(orc, setup, x):
    g, S, _, d, dd = setup
    h = orc.direct(x, W.T0_C1, MODES, g.f0, g.df, g.n_bins)
    dh, hh = orc.inner(d, h, S, g.df), orc.inner(h, h, S, g.df)
    return dh - 0.5 * hh - 0.5 * dd, dh, hh


def test_edges_cover_every_band(orc, setup):
    g, S, th, d, dd = setup
    e = R.edges(th, W.T0_C1, MODES, g, 64)
    assert np.all(np.diff(e) > 0)
    for (l, m) in MODES:
        b = orc.band(th, W.T0_C1, l, m, g.f0, g.df, g.n_bins)
        assert b[2] in e and b[3] + 1 in e
    assert e[0] == min(orc.band(th, W.T0_C1, l, m, g.f0, g.df, g.n_bins)[2] for l, m in MODES)


def test_summary_data_add_up_to_the_dense_inner_products(orc, setup):
    g, S, th, d, dd = setup
    e = R.edges(th, W.T0_C1, MODES, g, 64)
    A0, A1, B0, B1 = R.summary(th, W.T0_C1, MODES, g, e, d, S)
    for a, (l, m) in enumerate(MODES):
        h = orc.direct(th, W.T0_C1, [(l, m)], g.f0, g.df, g.n_bins)
        assert abs(A0[a].sum().real - orc.inner(d, h, S, g.df)) <= 1e-9 * dd
        assert abs(B0[a, a].sum().real - orc.inner(h, h, S, g.df)) <= 1e-9 * dd
    assert np.allclose(B0, np.conj(np.swapaxes(B0, 0, 1)), rtol=0, atol=1e-12 * dd)


def test_exact_at_the_fiducial_and_for_constant_ratios(orc, setup):
    g, S, th, d, dd = setup
    e = R.edges(th, W.T0_C1, MODES, g, 64)
    summ = R.summary(th, W.T0_C1, MODES, g, e, d, S)
    for x in (th, th * np.where(np.arange(11) == 4, 2.0, 1.0)):
        a = R.loglike(x, th, W.T0_C1, MODES, g, e, summ, dd)
        b = dense(orc, setup, x)
        assert abs(a[0] - b[0]) <= 1e-9 * dd and abs(a[2] - b[2]) <= 1e-9 * dd


def test_second_order_convergence_near_the_fiducial(orc, setup):
    """The linear ratio leaves an error O(bin width^2): doubling the bins divides it by
    about four; with 256 bins a walker ~1e-4 away (Delta ln L ~ 180) is within 0.05."""
    g, S, th, d, dd = setup
    x = th * (1 + 1e-4 * np.random.default_rng(1).standard_normal(11))
    ref = dense(orc, setup, x)[0]
    err = []
    for n in (64, 128, 256):
        e = R.edges(th, W.T0_C1, MODES, g, n)
        summ = R.summary(th, W.T0_C1, MODES, g, e, d, S)
        err.append(abs(R.loglike(x, th, W.T0_C1, MODES, g, e, summ, dd)[0] - ref))
    assert err[0] / err[1] > 3.0 and err[1] / err[2] > 3.0, err
    assert err[2] < 0.05
