"""The CUDA relative-binning likelihood (lisa_like_set_fiducial, lisa_like_loglike_rb)
against the oracle's relative binning on the same data and fiducial, and against the
dense likelihood it approximates."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle_rb as R

pytestmark = pytest.mark.gpu
MODES3 = [(2, 2), (3, 3), (4, 4)]


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2005_01827_gb300 import build

    build.build()
    import paper_2005_01827_gb300 as p

    return p


def c1_setup(orc):
    g = W.GRID_C1
    S = orc.psd_aet(g.freqs())
    th = np.array(W.THETA_C1_Z)
    th[4] = orc.dl_gpc(th[4])
    th[10] = 1000.0
    d = orc.direct(th, W.T0_C1, MODES3, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 3))
    return g, S, th, d, orc.inner(d, d, S, g.df)


@pytest.mark.parametrize("n_rb", [64, 256])
def test_matches_the_oracle_relative_binning(pkg, orc, n_rb):
    g, S, th, d, dd = c1_setup(orc)
    like = pkg.LisaLike(modes=MODES3, n_knots=128, t0=W.T0_C1, max_batch=16)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    like.set_fiducial(th, n_rb)
    e = R.edges(th, W.T0_C1, MODES3, g, n_rb)
    assert np.array_equal(like.rb_edges(), e)
    summ = R.summary(th, W.T0_C1, MODES3, g, e, d, S)
    rng = np.random.default_rng(4)
    X = th * (1 + 1e-4 * rng.standard_normal((16, 11)))
    X[0] = th                                           # the fiducial itself
    X[1] = th
    X[1, 4] *= 2.0                                      # a pure distance rescaling
    X[2, 1] = 1.5                                       # invalid (q > 1)
    lnL, dh, hh = like.loglike_rb(X)
    like.close()
    assert lnL[2] == -np.inf and dh[2] == 0.0
    for b in range(16):
        if b == 2:
            continue
        ref = R.loglike(X[b], th, W.T0_C1, MODES3, g, e, summ, dd)
        scale = max(dd, abs(ref[2]))
        assert abs(lnL[b] - ref[0]) <= 1e-9 * scale, (b, lnL[b], ref[0])
        assert abs(hh[b] - ref[2]) <= 1e-9 * scale
    # exact at the fiducial and under a distance rescaling: the dense direct likelihood
    for b in (0, 1):
        h = orc.direct(X[b], W.T0_C1, MODES3, g.f0, g.df, g.n_bins)
        dense = orc.inner(d, h, S, g.df) - 0.5 * orc.inner(h, h, S, g.df) - 0.5 * dd
        assert abs(lnL[b] - dense) <= 1e-9 * dd


def test_full_grid_six_modes_near_the_injection(pkg, orc):
    """The sampler workload's data (1-yr grid, six modes, SNR ~880): relative binning
    about the injection against the dense FP64 likelihood of the hot path for walkers at
    posterior-scale offsets."""
    g = W.GRID_C2
    S = orc.psd_aet(g.freqs())
    inj = np.array(W.THETA_SAMPLER_Z)
    inj[4] = orc.dl_gpc(inj[4])
    d = orc.template(inj, W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 2))
    like = pkg.LisaLike(modes=W.MODES6, n_knots=1024, max_batch=64)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    like.set_fiducial(inj, 256)
    rng = np.random.default_rng(7)
    X = inj * (1 + 2e-4 * rng.standard_normal((64, 11)))
    X[:, 1] = np.minimum(X[:, 1], 1.0)
    X[0] = inj
    lrb, _, hrb = like.loglike_rb(X)
    lden, _, hden = like.loglike(X)
    like.close()
    err = np.abs(lrb - lden)
    print("relative binning vs dense FP64 over 64 walkers: max |d lnL| %.3e, median %.3e, "
          "ln L spread %.1f" % (err.max(), np.median(err), lden.max() - lden.min()))
    assert np.all(np.isfinite(lrb))
    assert err.max() <= 0.5 and np.median(err) <= 0.05
    # the walkers' ranking by ln L (what a sampler uses) is preserved
    assert np.array_equal(np.argsort(lrb)[-10:], np.argsort(lden)[-10:])
