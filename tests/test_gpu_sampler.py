"""The CUDA sampler (include/lisa_sampler.h) against the oracle sampler on the same
seeded inputs: both sides draw the same Philox streams, so chains agree walker by walker
and step by step while every accept/reject decision agrees."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
D = 11
MEAN = np.linspace(-1.0, 1.0, D)
SIGMA = np.linspace(0.5, 2.0, D)
BOX_LO, BOX_HI = np.full(D, -60.0), np.full(D, 60.0)


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2005_01827_gb300 import build

    build.build()
    import paper_2005_01827_gb300 as p

    return p


def gauss_sampler(pkg, T, Wk, graphs, adaptive, seed=5):
    LL = pkg.lisalike
    return LL.LisaSampler(None, n_temps=T, n_walkers=Wk, a=2.0, target=LL.LISA_TARGET_GAUSSIAN,
                          gauss_mean=MEAN, gauss_sigma=SIGMA, lower=BOX_LO, upper=BOX_HI,
                          seed=seed, adaptive=int(adaptive), adapt_lag=50.0, adapt_time=5.0,
                          use_graphs=int(graphs), lisa_frame=0)


@pytest.mark.parametrize("graphs", [True, False])
def test_gaussian_chains_match_the_oracle(pkg, orc, graphs):
    T, Wk, n = 4, 32, 300
    betas = np.array([1.0, 0.6, 0.3, 0.0])
    rng = np.random.default_rng(3)
    x0 = MEAN + 2.0 * SIGMA * rng.standard_normal((T, Wk, D))
    s = gauss_sampler(pkg, T, Wk, graphs, True)
    s.set_ladder(betas)
    s.set_state(x0, step=7)
    ch1, l1 = s.run(n // 2)
    ch2, l2 = s.run(n - n // 2)
    x, lnl, b, step = s.state()
    acc, sw = s.counts()
    assert s.step_launches() == 5 and step == 7 + n
    s.close()
    r = orc.sampler_gauss(x0, betas, MEAN, SIGMA, n, 5, BOX_LO, BOX_HI, a=2.0, step0=7,
                          adaptive=True, adapt_lag=50.0, adapt_time=5.0)
    chain = np.concatenate([ch1, ch2])
    lch = np.concatenate([l1, l2])
    # identical arithmetic on both sides: equal unless a log() rounding flips a decision
    assert np.array_equal(chain, r.chain)
    assert np.array_equal(lch, r.lnl_chain)
    assert np.array_equal(x, r.x) and np.array_equal(lnl, r.lnl)
    assert np.array_equal(acc, r.acc) and np.array_equal(sw, r.swaps)
    assert np.allclose(b, r.betas, rtol=1e-13, atol=0)
    assert not np.array_equal(b, betas)                    # the ladder moved


def test_to_physical_matches_the_oracle(pkg, orc):
    import torch

    LL = pkg.lisalike
    rng = np.random.default_rng(4)
    n = 257
    x = np.column_stack([
        rng.uniform(W.TABLE1_LOWER[q], W.TABLE1_UPPER[q], n) for q in range(D)])
    dx = torch.tensor(x, dtype=torch.float64, device="cuda")
    out = torch.empty_like(dx)
    for frame in (0, 1):
        LL.lisa_sampler_to_physical(dx, n, frame, W.T0_YEAR, out)
        torch.cuda.synchronize()
        th = out.cpu().numpy()
        ref = np.array([orc.to_physical(v, bool(frame), W.T0_YEAR) for v in x])
        scale = np.maximum(np.abs(ref), 1.0)
        ang = np.abs(th - ref)
        ang[:, 7] = np.abs((th[:, 7] - ref[:, 7] + np.pi) % (2 * np.pi) - np.pi)
        ang[:, 9] = np.abs((th[:, 9] - ref[:, 9] + np.pi / 2) % np.pi - np.pi / 2)
        assert np.max(ang / scale) <= 1e-11, (frame, np.max(ang / scale, axis=0))


def test_autocorr_time_matches_the_oracle(pkg, orc):
    import torch

    LL = pkg.lisalike
    rng = np.random.default_rng(5)
    n, Wk, phi = 3000, 24, 0.8
    e = rng.standard_normal((n, Wk, 3))
    x = np.empty_like(e)
    x[0] = e[0]
    for i in range(1, n):
        x[i] = phi * x[i - 1] + e[i]
    dx = torch.tensor(x, dtype=torch.float64, device="cuda")
    for off in range(3):
        rho = np.empty(n)
        torch.cuda.synchronize()
        tau = LL.lisa_autocorr_time(dx, n, Wk, 3, off, rho)
        tr, rr = orc.autocorr_time(np.ascontiguousarray(x[:, :, off]), return_rho=True)
        assert abs(tau - tr) <= 1e-10 * tr
        assert np.max(np.abs(rho - rr)) <= 1e-12


def lisa_setup(orc, modes, K):
    g = W.GRID_C1
    S = orc.psd_aet(g.freqs())
    inj = np.array(W.THETA_C1_Z)
    inj[4] = orc.dl_gpc(inj[4])
    inj[10] = 1000.0      # beyond the largest Roemer delay (500 s): t_ref > 0 in both frames
    d = orc.template(inj, W.T0_C1, modes, K, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 6))
    return g, S, inj, d


@pytest.mark.parametrize("frame", [False, True])
def test_lisa_chains_match_the_oracle(pkg, orc, frame):
    """Sampler on the batched FP64 likelihood (two modes, 25661 bins) against the oracle
    sampler on the oracle likelihood: the same decisions, hence the same chains, and ln L
    within the FP64 parity bound."""
    LL = pkg.lisalike
    modes, K, T, Wk, n = [(2, 2), (3, 3)], 128, 2, 16, 6
    g, S, inj, d = lisa_setup(orc, modes, K)
    xc = orc.from_physical(inj)
    if frame:   # the same point in LISA-frame coordinates
        tL, lamL, betL, psiL = orc.ssb_to_lisa(inj[10] + W.T0_C1, inj[7], inj[8], inj[9])
        xc[7], xc[8], xc[9], xc[10] = lamL, math.sin(betL), psiL, math.log(tL - W.T0_C1)
    scale = np.array([1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-2, 1e-3, 1e-3, 1e-3, 1e-2, 1e-2])
    x0 = LL.sky_mode_init(xc, scale, W.TABLE1_LOWER, W.TABLE1_UPPER, T, Wk, 11)
    x0[:, 8:] = xc + scale * np.random.default_rng(1).standard_normal((T, Wk - 8, D))
    betas = [1.0, 0.25]
    like = pkg.LisaLike(modes=modes, n_knots=K, t0=W.T0_C1, max_batch=T * Wk // 2)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    s = LL.LisaSampler(like, n_temps=T, n_walkers=Wk, seed=9, lisa_frame=int(frame),
                       adaptive=0, t_max_inf=0, lower=W.TABLE1_LOWER, upper=W.TABLE1_UPPER)
    s.set_ladder(betas)
    s.set_state(x0)
    chain, lch = s.run(n)
    x, lnl, _, _ = s.state()
    acc, sw = s.counts()
    assert s.step_launches() == 2 * (1 + like.last_launches() + 1) + 1
    s.close()
    like.close()
    r = orc.sampler_lisa(x0, betas, n, 9, W.TABLE1_LOWER, W.TABLE1_UPPER, W.T0_C1, modes, K,
                         g.f0, g.df, d, S, lisa_frame=frame)
    assert np.array_equal(chain, r.chain)
    assert np.array_equal(acc, r.acc) and np.array_equal(sw, r.swaps)
    assert acc[0, 0] > 0
    snr2 = max(orc.inner(d, d, S, g.df), 1.0)
    fin = np.isfinite(r.lnl)
    assert np.array_equal(fin, np.isfinite(lnl))
    assert np.max(np.abs(lnl - r.lnl)[fin]) <= 1e-6 * snr2
    assert np.max(np.abs(lch - r.lnl_chain)) <= 1e-6 * snr2


def test_sampler_host_timeout_is_reported_and_recovers(pkg):
    """A host wait whose bound runs out returns LISA_ERR_TIMEOUT without any device
    fault; after the device is idle a new sampler runs normally."""
    import torch

    LL = pkg.lisalike
    rng = np.random.default_rng(2)
    x0 = MEAN + SIGMA * rng.standard_normal((8, 4096, D))
    s = None
    with pytest.raises(LL.LisaError) as e:   # the first wait that runs out: create, state or run
        s = LL.LisaSampler(None, n_temps=8, n_walkers=4096, target=LL.LISA_TARGET_GAUSSIAN,
                           gauss_mean=MEAN, gauss_sigma=SIGMA, lower=BOX_LO, upper=BOX_HI,
                           lisa_frame=0, timeout_s=1e-7)
        s.set_state(x0)
        s.run(50, record=False)
    assert e.value.status == LL.LISA_ERR_TIMEOUT
    torch.cuda.synchronize()
    if s is not None:
        s.close()
    s = gauss_sampler(pkg, 2, 8, True, False)
    s.set_state(x0[:2, :8])
    s.run(3)
    s.close()


def test_bad_configurations_are_rejected(pkg):
    LL = pkg.lisalike
    for kw in (dict(n_walkers=7), dict(n_walkers=2), dict(n_temps=0), dict(n_temps=65),
               dict(a=1.0), dict(ladder_ratio=0.5)):
        with pytest.raises(LL.LisaError) as e:
            LL.LisaSampler(None, target=LL.LISA_TARGET_GAUSSIAN, **kw)
        assert e.value.status == LL.LISA_ERR_ARG
    with pytest.raises(LL.LisaError):
        LL.LisaSampler(None)                      # the likelihood target needs a handle
    s = LL.LisaSampler(None, target=LL.LISA_TARGET_GAUSSIAN, n_temps=3, n_walkers=8)
    with pytest.raises(LL.LisaError) as e:
        s.run(1)                                  # no state yet
    assert e.value.status == LL.LISA_ERR_STATE
    with pytest.raises(LL.LisaError):
        s.set_ladder([1.0, 0.5, 0.7])             # increasing temperature index, rising beta
    s.close()


def sampler_workload(orc):
    """8 temperatures x 256 walkers on the 1-yr grid, 6 modes, around the M_T = 2e6,
    q = 0.5, z = 3 injection in noise; walkers start at the 8 LISA-frame sky modes."""
    g = W.GRID_C2
    S = orc.psd_aet(g.freqs())
    inj = np.array(W.THETA_SAMPLER_Z)
    inj[4] = orc.dl_gpc(inj[4])
    d = orc.template(inj, W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 2))
    xc = orc.from_physical(inj)
    tL, lamL, betL, psiL = orc.ssb_to_lisa(inj[10] + W.T0_YEAR, inj[7], inj[8], inj[9])
    xc[7], xc[8], xc[9], xc[10] = lamL, math.sin(betL), psiL, math.log(tL - W.T0_YEAR)
    return g, S, inj, d, xc


def test_sampler_workload_full_size(pkg, orc):
    """Graph-replayed steps of the full sampler workload: sampled walkers of every
    temperature carry the oracle ln L of their (LISA-frame-converted) parameters."""
    LL = pkg.lisalike
    g, S, inj, d, xc = sampler_workload(orc)
    T, Wk = W.SAMPLER_T, W.SAMPLER_W
    like = pkg.LisaLike(modes=W.MODES6, n_knots=1024, max_batch=T * Wk // 2)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    scale = np.full(D, 1e-3)
    x0 = LL.sky_mode_init(xc, scale, W.TABLE1_LOWER, W.TABLE1_UPPER, T, Wk, 5)
    s = LL.LisaSampler(like)                    # defaults: 8 x 256, a = 1.15, adaptive
    assert (s.T, s.W) == (T, Wk)
    s.set_state(x0)
    chain, lch = s.run(2)
    x, lnl, betas, step = s.state()
    acc, sw = s.counts()
    s.close()
    dd = like.data_inner()
    like.close()
    assert step == 2 and betas[0] == 1.0 and betas[-1] == 0.0
    assert np.array_equal(chain[-1], x[0]) and np.array_equal(lch[-1], lnl[0])
    assert acc[:, 1].tolist() == [2 * Wk] * T
    pick = [(0, 0), (0, 77), (2, 5), (4, 200), (6, 31), (7, 255)]
    th = np.array([orc.to_physical(x[t, w], True, W.T0_YEAR) for t, w in pick])
    ref, _, rhh, _ = orc.loglike(th, W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, d, S)
    got = np.array([lnl[t, w] for t, w in pick])
    scale_ = np.maximum(np.maximum(rhh, dd), 1.0)
    err = np.abs(got - ref) / scale_
    print("sampler workload sampled max |d lnL| / SNR^2 = %.3e" % err.max())
    assert np.all(err <= 1e-6)
    # the coldest walkers at the true sky mode sit near the injection's ln L
    assert np.max(lnl[0]) > -0.5 * dd + 0.5 * 880.0 ** 2 * 0.5


def test_checkpoint_resume_continues_the_same_chain(pkg, tmp_path):
    """Checkpoint/resume: 40 steps, save, a new sampler restores and runs 60 more; the
    chain equals 100 uninterrupted steps (the ladder adapts throughout)."""
    T, Wk = 3, 16
    rng = np.random.default_rng(8)
    x0 = MEAN + SIGMA * rng.standard_normal((T, Wk, D))
    s = gauss_sampler(pkg, T, Wk, True, True, seed=21)
    s.set_state(x0)
    full, _ = s.run(100)
    xf, _, bf, _ = s.state()
    s.close()
    s = gauss_sampler(pkg, T, Wk, True, True, seed=21)
    s.set_state(x0)
    a, _ = s.run(40)
    s.checkpoint(tmp_path / "ck.npz")
    s.close()
    s = gauss_sampler(pkg, T, Wk, False, True, seed=21)
    s.restore(tmp_path / "ck.npz")
    b, _ = s.run(60)
    xr, _, br, step = s.state()
    s.close()
    assert step == 100
    assert np.array_equal(np.concatenate([a, b]), full)
    assert np.array_equal(xr, xf) and np.array_equal(br, bf)
