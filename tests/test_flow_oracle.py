"""Pins of the oracle's normalizing-flow proposal: bfloat16 rounding against an
independent conversion, closed forms (identity flow, first Adam step), exact
invertibility, the log-determinant against a numerical Jacobian, back-propagation
against finite differences, learning a known correlated Gaussian, Box-Muller latent
draws, and the independence Metropolis-Hastings rule of Eq. (13) sampling its target
with a deliberately poor proposal."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle_flow as F

D = 11


def test_bf16_rounding_matches_an_independent_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.uniform(-8, 8, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(F.bf16(x), ref)


def gauss_setup(seed=0):
    rng = np.random.default_rng(seed)
    mu = rng.normal(size=D)
    sig = rng.uniform(0.5, 2.0, D)
    return rng, mu, sig


def test_identity_flow_is_the_standard_normal():
    rng, mu, sig = gauss_setup()
    w = W.flow_init_weights(1, out_scale=0.0)
    x = mu + sig * rng.normal(size=(50, D))
    z, lq = F.normalize(w, x, mu, sig)
    u = (x - mu) / sig
    want = -0.5 * np.sum(u * u, axis=1) - 0.5 * D * math.log(2 * math.pi) - np.sum(np.log(sig))
    assert np.allclose(z, u, atol=1e-15) and np.allclose(lq, want, atol=1e-12)


def test_generate_inverts_normalize_and_agrees_on_the_density():
    rng, mu, sig = gauss_setup(1)
    w = W.flow_init_weights(2, out_scale=0.2)
    x = mu + sig * rng.normal(size=(200, D))
    z, lq = F.normalize(w, x, mu, sig)
    x2, lq2 = F.generate(w, z, mu, sig)
    assert np.max(np.abs(x2 - x)) <= 1e-10
    assert np.max(np.abs(lq2 - lq)) <= 1e-9


def test_log_determinant_matches_the_numerical_jacobian():
    rng, mu, sig = gauss_setup(2)
    w = W.flow_init_weights(3, out_scale=0.2)
    for xi in mu + sig * rng.normal(size=(3, D)):
        J = np.zeros((D, D))
        h = 1e-6
        for d in range(D):
            e = np.zeros(D)
            e[d] = h
            J[:, d] = (F.normalize(w, (xi + e)[None], mu, sig, quant=False)[0][0]
                       - F.normalize(w, (xi - e)[None], mu, sig, quant=False)[0][0]) / (2 * h)
        z, lq = F.normalize(w, xi[None], mu, sig, quant=False)
        logdet = lq[0] + 0.5 * np.sum(z * z) + 0.5 * D * math.log(2 * math.pi)
        assert abs(np.linalg.slogdet(J)[1] - logdet) <= 1e-6


def test_backpropagation_matches_finite_differences():
    rng, mu, sig = gauss_setup(3)
    w = {k: v.astype(np.float64) for k, v in W.flow_init_weights(4, out_scale=0.2).items()}
    u = rng.normal(size=(32, D))
    _, g = F.nll_grads(w, u, quant=False)
    picks = {"W1": [(0, 3, 2), (5, 100, 7)], "b1": [(2, 17)], "W2": [(1, 5, 6), (7, 127, 0)],
             "b2": [(3, 64)], "W3": [(0, 2, 9), (6, 15, 100)], "b3": [(4, 1), (7, 20)]}
    for k, idxs in picks.items():
        for idx in idxs:
            wp = {kk: vv.copy() for kk, vv in w.items()}
            wm = {kk: vv.copy() for kk, vv in w.items()}
            eps = 1e-6
            wp[k][idx] += eps
            wm[k][idx] -= eps
            num = (F.nll_grads(wp, u, quant=False)[0] - F.nll_grads(wm, u, quant=False)[0]) / (2 * eps)
            assert abs(g[k][idx] - num) <= 1e-6 * max(1.0, abs(num)), (k, idx, g[k][idx], num)


def test_first_adam_step_is_a_signed_learning_rate():
    w = W.flow_init_weights(5, out_scale=0.1)
    rng = np.random.default_rng(4)
    g = {k: rng.normal(size=v.shape) for k, v in w.items()}
    w2, _ = F.adam(w, g, F.adam_state(w), 1e-3)
    for k in w:
        step = w[k].astype(np.float64) - w2[k].astype(np.float64)
        # bias-corrected moments at t = 1 are g and g^2: the step is lr g / (|g| + eps)
        assert np.allclose(step, 1e-3 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-4, atol=1e-9)


def correlated_gaussian(seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(D, D))
    cov = A @ A.T / D + 0.05 * np.eye(D)
    return rng, rng.normal(size=D), cov, np.linalg.cholesky(cov)


def test_whitening_alone_fits_a_correlated_gaussian():
    """With u = L^{-1}(x - mu) from the sample covariance, the identity flow is the
    Gaussian fit: held-out NLL at the exact entropy; whitening recovers mean and
    covariance."""
    rng, mu, cov, L = correlated_gaussian(0)
    data = mu + rng.normal(size=(20000, D)) @ L.T
    test = mu + rng.normal(size=(4000, D)) @ L.T
    H = 0.5 * np.linalg.slogdet(2 * np.pi * np.e * cov)[1]
    m, Lw = F.whitening(data)
    assert np.allclose(Lw @ Lw.T, np.cov(data.T, bias=True), rtol=1e-10, atol=1e-12)
    assert np.allclose(np.triu(Lw, 1), 0.0)
    nll0 = -F.normalize(W.flow_init_weights(3, 0.0), test, m, Lw)[1].mean()
    assert abs(nll0 - H) < 0.05, (nll0, H)


def banana(n, rng, A):
    """x1 = x0^2 + N(0, 1/4), the other coordinates standard normal, then mixed by A:
    entropy (D/2) log(2 pi e) + log(1/2) + log|det A| exactly (x1 - x0^2 preserves
    volume)."""
    z = rng.normal(size=(n, D))
    z[:, 1] = z[:, 0] ** 2 + 0.5 * z[:, 1]
    return z @ A.T


def test_training_learns_a_banana():
    """Held-out NLL within 0.3 nats of the exact entropy after 300 BF16 Adam steps; the
    whitened identity flow (a Gaussian fit) is more than 0.8 nats worse."""
    rng = np.random.default_rng(0)
    A = rng.normal(size=(D, D)) / math.sqrt(D) + np.eye(D)
    H = 0.5 * D * math.log(2 * math.pi * math.e) + math.log(0.5) + np.linalg.slogdet(A)[1]
    data, test = banana(20000, rng, A), banana(4000, rng, A)
    w0 = W.flow_init_weights(3, 0.0)
    w, m, L, losses = F.train(w0, data, 300, 256, 2e-3, F.minibatch_index(7))
    nll = -F.normalize(w, test, m, L)[1].mean()
    nll0 = -F.normalize(w0, test, m, L)[1].mean()
    assert nll - H < 0.3 and nll0 - H > 0.8, (nll, nll0, H)
    assert losses[-20:].mean() < losses[:20].mean() - 0.5


def test_latent_draws_are_standard_normal():
    z = F.latent_draws(123, 5, range(1500)).ravel()
    assert abs(z.mean()) < 4.0 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4.0 * math.sqrt(2.0 / z.size)
    from scipy import stats

    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_independence_mh_samples_the_target_with_a_poor_proposal():
    """Eq. (13) with the q(x)/q(y) factor: a proposal that is shifted, too narrow and
    distorted still leaves the target N(mu, diag sigma^2) invariant."""
    mu_t = np.linspace(-1.0, 1.0, D)
    sig_t = np.linspace(0.5, 1.5, D)
    w = W.flow_init_weights(8, out_scale=0.15)
    mu_q, sig_q = mu_t + 0.3 * sig_t, 0.8 * sig_t
    lo, hi = np.full(D, -50.0), np.full(D, 50.0)

    def target(y):
        r = (y - mu_t) / sig_t
        return -0.5 * np.sum(r * r, axis=1)

    rng = np.random.default_rng(9)
    x = mu_t + sig_t * rng.normal(size=(64, D))
    lnl, lnp = target(x), np.zeros(64)
    chain, n_acc = [], 0
    for step in range(1500):
        x, lnl, lnp, acc, _ = F.flow_mh_step(w, mu_q, sig_q, x, lnl, lnp, 1.0, 77, step, lo, hi,
                                             target)
        n_acc += acc.sum()
        chain.append(x.copy())
    ch = np.array(chain[100:])
    flat = ch.reshape(-1, D)
    from test_sampler_oracle import tau_fft

    tau = np.array([tau_fft(ch[:, :, q])[0] for q in range(D)])
    n_eff = ch.shape[0] * ch.shape[1] / tau
    zm = (flat.mean(axis=0) - mu_t) / (sig_t / np.sqrt(n_eff))
    zv = (flat.var(axis=0) / sig_t ** 2 - 1.0) / np.sqrt(2.0 / n_eff)
    assert np.max(np.abs(zm)) < 4.5 and np.max(np.abs(zv)) < 4.5, (zm, zv)
    assert 0.05 < n_acc / (1500 * 64) < 0.95
