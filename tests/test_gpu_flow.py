"""The CUDA normalizing flow (include/lisa_flow.h) and its use as an independence
proposal in the sampler, against the numpy oracle (oracle/oracle_flow.py).

The device runs the networks with bfloat16 operands and FP32 accumulation; the oracle
rounds the same operands to bfloat16 and accumulates exactly.  Rounding differences of
the accumulations occasionally move an operand across a bfloat16 boundary (a relative
step of 2^-8), so outputs are compared by quantiles: most samples agree to FP32
accuracy and every sample within the effect of such a step."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle_flow as F

pytestmark = pytest.mark.gpu
D = 11


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2005_01827_gb300 import build

    build.build()
    import paper_2005_01827_gb300 as p

    return p


def setup_flow(pkg, seed=3, out_scale=0.3):
    rng = np.random.default_rng(seed)
    mu = rng.normal(size=D)
    sig = rng.uniform(0.5, 2.0, D)
    w = W.flow_init_weights(seed, out_scale=out_scale)
    fl = pkg.lisalike.Flow(seed=1)
    fl.set_weights(w)
    fl.set_standardisation(mu, sig)
    return rng, mu, sig, w, fl


def test_weights_round_trip(pkg):
    _, _, _, w, fl = setup_flow(pkg)
    back = fl.weights()
    for k in w:
        assert np.array_equal(back[k], w[k]), k
    fl.close()


def test_normalize_and_generate_match_the_oracle(pkg):
    """FP32 errors scale with the size of log q (|z|^2 / 2): compare relative to it."""
    rng, mu, sig, w, fl = setup_flow(pkg, out_scale=0.1)
    n = 4099                                           # 65 blocks, ragged last block
    x = mu + sig * rng.normal(size=(n, D))
    z, lq = fl.normalize(x)
    zr, lqr = F.normalize(w, x, mu, sig)
    dq = np.abs(lq - lqr) / (1.0 + np.abs(lqr))
    dz = np.max(np.abs(z - zr), axis=1) / np.maximum(1.0, np.max(np.abs(zr), axis=1))
    print("normalize rel |d log q| quantiles 50/95/100: %.2e %.2e %.2e" % tuple(np.quantile(dq, [0.5, 0.95, 1.0])))
    print("normalize rel |d z| quantiles 50/95/100: %.2e %.2e %.2e" % tuple(np.quantile(dz, [0.5, 0.95, 1.0])))
    assert np.quantile(dq, 0.95) <= 1e-5 and dq.max() <= 1e-2
    assert np.quantile(dz, 0.95) <= 1e-5 and dz.max() <= 1e-2
    x2, lq2 = fl.generate(zr)
    xr, lqr2 = F.generate(w, zr, mu, sig)
    dx = np.max(np.abs(x2 - xr) / sig, axis=1) / np.maximum(1.0, np.max(np.abs(zr), axis=1))
    dq2 = np.abs(lq2 - lqr2) / (1.0 + np.abs(lqr2))
    print("generate rel |d x| quantiles 50/95/100: %.2e %.2e %.2e" % tuple(np.quantile(dx, [0.5, 0.95, 1.0])))
    assert np.quantile(dx, 0.95) <= 1e-5 and dx.max() <= 1e-2
    assert np.quantile(dq2, 0.95) <= 1e-5 and dq2.max() <= 1e-2
    # the device round trip is exact up to FP32
    x3, _ = fl.generate(z)
    assert np.quantile(np.max(np.abs(x3 - x) / sig, axis=1), 0.99) <= 1e-4
    fl.close()


def test_gradients_match_the_oracle(pkg):
    rng, mu, sig, w, fl = setup_flow(pkg, 5, 0.2)
    x = mu + sig * rng.normal(size=(512, D))
    loss, g = fl.gradients(x)
    lr_, gr = F.nll_grads(w, F.whiten(x, mu, sig))
    assert abs(loss - lr_) <= 1e-4 * max(1.0, abs(lr_))
    for k in g:
        rel = np.linalg.norm(g[k] - gr[k]) / max(np.linalg.norm(gr[k]), 1e-30)
        print("grad %s relative error %.2e" % (k, rel))
        assert rel <= 2e-2, k
    fl.close()


def test_training_learns_a_banana(pkg):
    """The device trainer reaches the oracle trainer's held-out NLL (both within 0.3 nats
    of the exact entropy of a non-Gaussian target) from the same start and minibatches,
    and its whitening equals the oracle's."""
    import torch
    from test_flow_oracle import banana

    rng = np.random.default_rng(0)
    A = rng.normal(size=(D, D)) / math.sqrt(D) + np.eye(D)
    H = 0.5 * D * math.log(2 * math.pi * math.e) + math.log(0.5) + np.linalg.slogdet(A)[1]
    data, test = banana(20000, rng, A), banana(4000, rng, A)
    w0 = W.flow_init_weights(3, 0.0)
    fl = pkg.lisalike.Flow(seed=1)
    fl.set_weights(w0)
    losses = fl.train(torch.tensor(data, device="cuda"), 300, batch=256, lr=2e-3, seed=7)
    m, L = fl.whitening()
    mo_, Lo_ = F.whitening(data)
    assert np.allclose(m, mo_, rtol=0, atol=1e-12)
    assert np.allclose(L, Lo_, rtol=1e-10, atol=1e-13)
    nll = -fl.normalize(test)[1].mean()
    wo, mo, Lo, lo = F.train(w0, data, 300, 256, 2e-3, F.minibatch_index(7))
    nll_o = -F.normalize(wo, test, mo, Lo)[1].mean()
    print("held-out NLL: device %.4f oracle %.4f entropy %.4f" % (nll, nll_o, H))
    assert nll - H < 0.3 and abs(nll - nll_o) < 0.1
    assert abs(losses[:5].mean() - lo[:5].mean()) < 1e-2     # same minibatches at the start
    fl.close()


def test_flow_mh_step_matches_the_oracle(pkg):
    """Flow-only sampler steps on a Gaussian target against the oracle's step from the
    same state: proposals agree to FP32 accuracy and decisions agree except where the
    log acceptance ratio lies within 1e-3 of ln u."""
    LL = pkg.lisalike
    mu_t = np.linspace(-1.0, 1.0, D)
    sig_t = np.linspace(0.5, 1.5, D)
    lo, hi = np.full(D, -50.0), np.full(D, 50.0)
    w = W.flow_init_weights(8, out_scale=0.15)
    mu_q, sig_q = mu_t + 0.3 * sig_t, 0.8 * sig_t
    s = LL.LisaSampler(None, n_temps=1, n_walkers=128, target=LL.LISA_TARGET_GAUSSIAN,
                       gauss_mean=mu_t, gauss_sigma=sig_t, lower=lo, upper=hi, seed=77,
                       lisa_frame=0)
    fl = s.enable_flow(train_every=0, flow_only=1)
    fl.set_weights(w)
    fl.set_standardisation(mu_q, sig_q)
    rng = np.random.default_rng(9)
    s.set_state((mu_t + sig_t * rng.normal(size=(128, D)))[None])

    def target(y):
        r = (y - mu_t) / sig_t
        return -0.5 * np.sum(r * r, axis=1)

    n_mismatch = n_acc = 0
    for step in range(12):
        x, lnl, _, st = s.state()
        s.run(1)
        x2, lnl2, _, _ = s.state()
        xo, lo_, po, acc, lr = F.flow_mh_step(w, mu_q, sig_q, x[0], lnl[0], np.zeros(128), 1.0,
                                              77, st, lo, hi, target)
        gacc = ~np.all(x2[0] == x[0], axis=1)
        u = F.accept_units(77, st, range(128))
        bad = gacc != acc
        assert np.all(np.abs(np.log(u[bad]) - lr[bad]) < 1e-3)
        n_mismatch += bad.sum()
        both = gacc & acc
        dxs = np.max(np.abs(x2[0][both] - xo[both]) / sig_t, axis=1)
        assert np.median(dxs) <= 1e-5 and np.max(dxs, initial=0.0) <= 5e-3
        assert np.max(np.abs(lnl2[0][both] - lo_[both]), initial=0.0) <= 1e-2
        n_acc += gacc.sum()
    facc, _, _ = s.flow_stats()
    assert facc[1] == 12 * 128 and facc[0] == n_acc
    assert n_mismatch <= 2 and n_acc > 100
    s.close()


def test_trained_flow_sampler_mixes_faster_on_a_gaussian(pkg):
    """PT sampler with flow proposals trained on its own coldest chain: the target's
    moments are recovered, the flow is accepted often, and the coldest chain's
    autocorrelation time drops well below the stretch-only sampler's."""
    LL = pkg.lisalike
    mu_t = np.linspace(-1.0, 1.0, D)
    sig_t = np.linspace(0.5, 2.0, D)
    lo, hi = np.full(D, -60.0), np.full(D, 60.0)
    rng = np.random.default_rng(4)
    x0 = mu_t + sig_t * rng.normal(size=(4, 256, D))
    taus = {}
    for use_flow in (False, True):
        s = LL.LisaSampler(None, n_temps=4, n_walkers=256, target=LL.LISA_TARGET_GAUSSIAN,
                           gauss_mean=mu_t, gauss_sigma=sig_t, lower=lo, upper=hi, seed=5,
                           lisa_frame=0, a=1.15, adaptive=0)
        s.set_ladder([1.0, 0.5, 0.25, 0.0])
        if use_flow:
            s.enable_flow(train_every=500, train_iters=300, batch=1024, lr=1e-3, seed=3,
                          freeze_after=1000)
        s.set_state(x0)
        s.run(1000, record=False)                     # burn-in; the flow trains at 500, 1000
        chain, _ = s.run(2000)
        if use_flow:
            facc, n_tr, loss = s.flow_stats()
            print("flow acceptance %.3f, last loss %.3f" % (facc[0] / facc[1], loss))
            assert n_tr == 2 and np.isfinite(loss)
            assert facc[0] / facc[1] > 0.3, facc
        s.close()
        flat = chain.reshape(-1, D)
        from test_sampler_oracle import tau_fft

        tau = np.array([tau_fft(chain[:, :, q])[0] for q in range(D)])
        n_eff = chain.shape[0] * chain.shape[1] / tau
        zm = (flat.mean(axis=0) - mu_t) / (sig_t / np.sqrt(n_eff))
        zv = (flat.var(axis=0) / sig_t ** 2 - 1.0) / np.sqrt(2.0 / n_eff)
        print("flow=%s tau max %.1f |zm| %.2f |zv| %.2f" % (use_flow, tau.max(), np.abs(zm).max(),
                                                            np.abs(zv).max()))
        assert np.max(np.abs(zm)) < 5.0 and np.max(np.abs(zv)) < 5.0
        taus[use_flow] = tau.max()
    assert taus[True] < 0.25 * taus[False], taus


def test_flow_moves_with_an_fp64_likelihood_match_the_oracle(pkg, orc):
    """A split-precision sampler whose flow moves are evaluated by an FP64 handle
    (exact acceptances): flow-only steps on the LISA likelihood (two modes, 25,661 bins)
    against the oracle's flow step on the oracle likelihood from the same state."""
    LL = pkg.lisalike
    modes, K = [(2, 2), (3, 3)], 128
    g = W.GRID_C1
    S = orc.psd_aet(g.freqs())
    inj = np.array(W.THETA_C1_Z)
    inj[4] = orc.dl_gpc(inj[4])
    inj[10] = 1000.0
    d = orc.template(inj, W.T0_C1, modes, K, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 6))
    xc = orc.from_physical(inj)
    lo, hi = W.TABLE1_LOWER, W.TABLE1_UPPER
    Wn = 64
    rng = np.random.default_rng(3)
    sig = np.array([1e-4, 1e-4, 1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-4, 1e-4, 1e-3, 1e-4])
    x0 = xc + sig * rng.standard_normal((Wn, D))
    like = pkg.LisaLike(modes=modes, n_knots=K, t0=W.T0_C1, max_batch=Wn, precision=1)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    like64 = pkg.LisaLike(modes=modes, n_knots=K, t0=W.T0_C1, max_batch=Wn, precision=0)
    like64.set_data(g.f0, g.df, g.n_bins, d, S)
    s = LL.LisaSampler(like, n_temps=1, n_walkers=Wn, seed=13, lisa_frame=0, lower=lo, upper=hi)
    fl = s.enable_flow(train_every=0, flow_only=1)
    s.set_flow_likelihood(like64)
    w = W.flow_init_weights(4, out_scale=0.05)
    mu_q, L_q = xc, np.diag(1.5 * sig)
    fl.set_weights(w)
    fl.set_whitening(mu_q, L_q)
    s.set_state(x0[None])

    def target(y):
        th = np.array([orc.to_physical(v, False, W.T0_C1) for v in y])
        return orc.loglike(th, W.T0_C1, modes, K, g.f0, g.df, d, S)[0]

    snr2 = orc.inner(d, d, S, g.df)
    n_acc = n_bad = 0
    for _ in range(3):
        x, lnl, _, st = s.state()
        lnl_o = target(x[0])                          # the state's ln L on the oracle
        s.run(1)
        x2, lnl2, _, _ = s.state()
        xo, lo_, _, acc, lr = F.flow_mh_step(w, mu_q, L_q, x[0], lnl_o, np.zeros(Wn), 1.0, 13,
                                             st, lo, hi, target)
        gacc = ~np.all(x2[0] == x[0], axis=1)
        u = F.accept_units(13, st, range(Wn))
        bad = gacc != acc
        assert np.all(np.abs(np.log(u[bad]) - lr[bad]) < 1e-3)
        n_bad += bad.sum()
        n_acc += gacc.sum()
        both = gacc & acc
        # accepted walkers carry the FP64 ln L of their new position
        assert np.max(np.abs(lnl2[0][both] - lo_[both]), initial=0.0) <= 1e-6 * snr2
    s.close()
    like.close()
    like64.close()
    assert n_acc > 0 and n_bad <= 2


def test_screened_flow_moves_equal_the_fp64_ones(pkg, orc):
    """Flow moves screened by the split-precision likelihood (margin 0.05 in ln L) give the
    same chain, bit for bit, as flow moves all evaluated by the FP64 handle: every
    proposal the screen does not reject is decided on its FP64 ln L, and the ones it
    rejects lie further below log u than the two precisions differ.  The FP64 handle then
    evaluates only the proposals sent on."""
    LL = pkg.lisalike
    modes, K = [(2, 2), (3, 3)], 128
    g = W.GRID_C1
    S = orc.psd_aet(g.freqs())
    inj = np.array(W.THETA_C1_Z)
    inj[4] = orc.dl_gpc(inj[4])
    inj[10] = 1000.0
    d = orc.template(inj, W.T0_C1, modes, K, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 6))
    xc = orc.from_physical(inj)
    lo, hi = W.TABLE1_LOWER, W.TABLE1_UPPER
    Wn, n_steps = 64, 8
    rng = np.random.default_rng(3)
    sig = np.array([1e-4, 1e-4, 1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-4, 1e-4, 1e-3, 1e-4])
    x0 = xc + sig * rng.standard_normal((Wn, D))
    like = pkg.LisaLike(modes=modes, n_knots=K, t0=W.T0_C1, max_batch=Wn, precision=1)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    like64 = pkg.LisaLike(modes=modes, n_knots=K, t0=W.T0_C1, max_batch=Wn, precision=0)
    like64.set_data(g.f0, g.df, g.n_bins, d, S)
    w = W.flow_init_weights(4, out_scale=0.05)

    def make(screen):
        s = LL.LisaSampler(like, n_temps=1, n_walkers=Wn, seed=13, lisa_frame=0, lower=lo,
                           upper=hi)
        fl = s.enable_flow(train_every=0, flow_only=1)
        if screen:
            with pytest.raises(LL.LisaError) as e:     # a screen needs a second likelihood
                s.set_flow_screen(0.05)
            assert e.value.status == LL.LISA_ERR_STATE
        s.set_flow_likelihood(like64)
        if screen:
            with pytest.raises(LL.LisaError) as e:
                s.set_flow_screen(-1.0)
            assert e.value.status == LL.LISA_ERR_ARG
            s.set_flow_screen(0.05)
        fl.set_weights(w)
        fl.set_whitening(xc, np.diag(1.5 * sig))
        s.set_state(x0[None])
        return s

    a, b = make(False), make(True)
    for _ in range(n_steps):
        a.run(1)
        b.run(1)
        xa, la, _, _ = a.state()
        xb, lb, _, _ = b.state()
        assert np.array_equal(xa, xb) and np.array_equal(la, lb)
    acc_a, acc_b = a.flow_stats()[0], b.flow_stats()[0]
    sent = b.flow_screen_count()
    print("screened flow moves: %d of %d proposals sent to the FP64 likelihood, %d accepted"
          % (sent, n_steps * Wn, acc_b[0]))
    assert np.array_equal(acc_a, acc_b) and acc_b[0] > 0
    assert acc_b[0] <= sent < n_steps * Wn
    a.close()
    b.close()
    like.close()
    like64.close()
