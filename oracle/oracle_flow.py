"""Plain numpy reference of the normalizing-flow proposal (TEST INFRASTRUCTURE ONLY:
only tests/ and bench.py's baseline legs use it; it shares no code with the CUDA path).

The flow is not part of the paper: it is an independence proposal for the
Metropolis-Hastings rule of Eq. (13), whose acceptance min(1, L(y)/L(x) Q(x)/Q(y))
keeps the chain exact for any proposal density Q.  Definitions written out here:

* Whitening u = L^{-1} (x - mu), mu the mean and L L^T the covariance of the training
  set (Cholesky factor, each pivot floored at 1e-12 of its diagonal entry); a vector
  sigma stands for L = diag(sigma).
* Eight affine coupling layers.  Layer c keeps the coordinates with mask m_c = 1 and
  maps the others: v = m u + (1 - m) (u - t) e^{-s}, with s = (1 - m) S tanh(o_s / S),
  t = (1 - m) o_t, S = 2, and (o_s, o_t) = W3 relu(W2 relu(W1 (m u) + b1) + b2) + b3
  (11 -> 128 -> 128 -> 22).  log |dv/du| = -sum s.  Masks: c mod 4 = 0 keeps the even
  coordinates, 1 the odd ones, 2 coordinates 0..5, 3 coordinates 6..10.
* Density: z = layers(u), log q(x) = -|z|^2/2 - (D/2) log 2 pi + sum_c log|det_c|
  - sum_d log L_dd.  Sampling runs the layers backwards from z ~ N(0, I):
  u = m v + (1 - m) (v e^{s} + t), s and t from m v (= m u).
* BF16 arithmetic of the networks: every GEMM operand (weights, layer inputs, hidden
  activations and, in training, the back-propagated gradients) is rounded to bfloat16
  (round to nearest even); products and sums are exact here (FP64), where the device
  accumulates in FP32.
* Training minimises the mean of -log q_u(u) over minibatches with Adam
  (Kingma & Ba 2015; beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on FP32 master weights.
"""
from __future__ import annotations

import math

import numpy as np

D, H, C = 11, 128, 8
S_MAX = 2.0


def masks() -> np.ndarray:
    m = np.zeros((C, D))
    d = np.arange(D)
    for c in range(C):
        m[c] = [(d % 2 == 0), (d % 2 == 1), (d < 6), (d >= 6)][c % 4]
    return m


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _q(x, on):
    return bf16(x) if on else np.asarray(x, dtype=np.float64)


def mlp(w, c, u, m, quant=True):
    """Outputs s, t of coupling c for layer inputs u [n, D], and the cache of the
    forward pass (the GEMM operands as the device sees them)."""
    W1, W2, W3 = (_q(w[k][c], quant) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (np.asarray(w[k][c], dtype=np.float64) for k in ("b1", "b2", "b3"))
    a0 = _q(u * m, quant)
    z1 = a0 @ W1.T + b1
    a1 = _q(np.maximum(z1, 0.0), quant)
    z2 = a1 @ W2.T + b2
    a2 = _q(np.maximum(z2, 0.0), quant)
    o = a2 @ W3.T + b3
    th = np.tanh(o[:, :D] / S_MAX)
    s = (1.0 - m) * S_MAX * th
    t = (1.0 - m) * o[:, D:]
    return s, t, (a0, z1, a1, z2, a2, th)


def as_factor(sig):
    """The whitening factor L (lower triangular) from a factor or a vector of scales."""
    sig = np.asarray(sig, dtype=np.float64)
    return np.diag(sig) if sig.ndim == 1 else sig


def whiten(x, mu, sig):
    """u = L^{-1} (x - mu) by forward substitution, rows of x."""
    L = as_factor(sig)
    y = np.asarray(x, dtype=np.float64) - mu
    u = np.zeros_like(y)
    for d in range(D):
        u[:, d] = (y[:, d] - u[:, :d] @ L[d, :d]) / L[d, d]
    return u


def normalize(w, x, mu, sig, quant=True):
    """x [n, D] -> z [n, D] and log q(x) [n]."""
    m = masks()
    u = whiten(x, mu, sig)
    logdet = np.zeros(u.shape[0])
    for c in range(C):
        s, t, _ = mlp(w, c, u, m[c], quant)
        u = m[c] * u + (1.0 - m[c]) * (u - t) * np.exp(-s)
        logdet -= s.sum(axis=1)
    logq = -0.5 * np.sum(u * u, axis=1) - 0.5 * D * math.log(2 * math.pi) + logdet
    return u, logq - np.sum(np.log(np.diag(as_factor(sig))))


def generate(w, z, mu, sig, quant=True):
    """z [n, D] -> x [n, D] and log q(x) [n]."""
    m = masks()
    v = np.asarray(z, dtype=np.float64)
    logq = -0.5 * np.sum(v * v, axis=1) - 0.5 * D * math.log(2 * math.pi)
    for c in reversed(range(C)):
        s, t, _ = mlp(w, c, v, m[c], quant)
        v = m[c] * v + (1.0 - m[c]) * (v * np.exp(s) + t)
        logq -= s.sum(axis=1)
    L = as_factor(sig)
    return mu + v @ L.T, logq - np.sum(np.log(np.diag(L)))


def nll_grads(w, u, quant=True):
    """Mean of -log q_u(u) (without the constant) over the batch u [n, D] and its
    gradients with respect to every weight and bias (back-propagation written out)."""
    m = masks()
    n = u.shape[0]
    ins = []
    cur = np.asarray(u, dtype=np.float64)
    loss = np.zeros(n)
    for c in range(C):
        ins.append(cur)
        s, t, _ = mlp(w, c, cur, m[c], quant)
        cur = m[c] * cur + (1.0 - m[c]) * (cur - t) * np.exp(-s)
        loss += s.sum(axis=1)
    loss += 0.5 * np.sum(cur * cur, axis=1)
    grads = {k: np.zeros(v.shape, dtype=np.float64) for k, v in w.items()}
    gv = cur / n                                  # d(mean loss)/dz
    for c in reversed(range(C)):
        uc = ins[c]
        mc = m[c]
        s, t, (a0, z1, a1, z2, a2, th) = mlp(w, c, uc, mc, quant)
        e = np.exp(-s)
        v = mc * uc + (1.0 - mc) * (uc - t) * e
        gs = (1.0 - mc) * (-gv * v + 1.0 / n)     # dL/ds (the log-det term gives 1/n)
        gt = (1.0 - mc) * (-gv * e)
        go = np.concatenate([gs * (1.0 - th * th), gt], axis=1)
        W1, W2, W3 = (_q(w[k][c], quant) for k in ("W1", "W2", "W3"))
        goq = _q(go, quant)
        grads["W3"][c] = goq.T @ a2
        grads["b3"][c] = go.sum(axis=0)
        g2 = (goq @ W3) * (z2 > 0)
        g2q = _q(g2, quant)
        grads["W2"][c] = g2q.T @ a1
        grads["b2"][c] = g2.sum(axis=0)
        g1 = (g2q @ W2) * (z1 > 0)
        g1q = _q(g1, quant)
        grads["W1"][c] = g1q.T @ a0
        grads["b1"][c] = g1.sum(axis=0)
        ga0 = g1q @ W1
        gv = mc * (gv + ga0) + (1.0 - mc) * gv * e
    return float(loss.mean()), grads


def adam(w, g, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on FP32 master weights; state = (t, m, v)."""
    t, mm, vv = state
    t += 1
    out = {}
    for k in w:
        mm[k] = b1 * mm[k] + (1 - b1) * g[k]
        vv[k] = b2 * vv[k] + (1 - b2) * g[k] * g[k]
        mh = mm[k] / (1 - b1 ** t)
        vh = vv[k] / (1 - b2 ** t)
        out[k] = (w[k] - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32)
    return out, (t, mm, vv)


def adam_state(w):
    return (0, {k: np.zeros(v.shape) for k, v in w.items()},
            {k: np.zeros(v.shape) for k, v in w.items()})


def whitening(x):
    """Mean and Cholesky factor of the (population) covariance of the rows of x."""
    x = np.asarray(x, dtype=np.float64)
    mu = x.mean(axis=0)
    C = (x - mu).T @ (x - mu) / x.shape[0]
    L = np.zeros((D, D))
    for i in range(D):
        for j in range(i + 1):
            acc = C[i, j] - L[i, :j] @ L[j, :j]
            if i == j:
                floor = 1e-12 * C[i, i] if C[i, i] > 0 else 1e-300
                L[i, i] = math.sqrt(max(acc, floor))
            else:
                L[i, j] = acc / L[j, j]
    return mu, L


def train(w, data, n_iter, batch, lr, index_fn, quant=True):
    """Adam on minibatches data[index_fn(i)]; returns weights, whitening, losses."""
    mu, L = whitening(data)
    u = whiten(data, mu, L)
    st = adam_state(w)
    losses = []
    for i in range(n_iter):
        loss, g = nll_grads(w, u[index_fn(i, batch, data.shape[0])], quant)
        w, st = adam(w, g, st, lr)
        losses.append(loss)
    return w, mu, L, np.array(losses)


# ----------------------------------------------------------------- proposal and MH step

def _philox_units(seed, ctr):
    from oracle import philox

    o = philox(ctr, (seed & 0xFFFFFFFF, seed >> 32))
    return (o.astype(np.float64) + 0.5) / 4294967296.0


def latent_draws(seed, step, walkers):
    """z [W, D]: twelve uniforms per walker from Philox counters (step, 3, blk, w),
    blk = 0..2, turned into normals by the Box-Muller transform in pairs
    (u_{2p}, u_{2p+1}); the first 11 of the 12 normals are used."""
    z = np.empty((len(walkers), D))
    for i, w in enumerate(walkers):
        u = np.concatenate([_philox_units(seed, (step, 3, blk, w)) for blk in range(3)])
        nrm = []
        for p in range(6):
            r = math.sqrt(-2.0 * math.log(u[2 * p]))
            nrm += [r * math.cos(2.0 * math.pi * u[2 * p + 1]),
                    r * math.sin(2.0 * math.pi * u[2 * p + 1])]
        z[i] = nrm[:D]
    return z


def accept_units(seed, step, walkers):
    return np.array([_philox_units(seed, (step, 4, 0, w))[0] for w in walkers])


def prior_ln(x, lo, hi):
    ok = np.all((x >= lo) & (x <= hi), axis=1)
    return np.where(ok, 0.0, -np.inf)


def flow_mh_step(wts, mu, sig, x, lnl, lnp, beta, seed, step, lo, hi, target):
    """Independence Metropolis-Hastings (Eq. (13)) for the walkers x [W, D] of one
    temperature: y = flow(z), accepted with probability
    min(1, [L(y)/L(x)]^beta pi(y)/pi(x) q(x)/q(y)).  target(y) -> ln L for points inside
    the prior.  Returns new (x, lnl, lnp), the acceptance mask and the log ratio."""
    Wn = x.shape[0]
    z = latent_draws(seed, step, range(Wn))
    y, qy = generate(wts, z, mu, sig)
    _, qx = normalize(wts, x, mu, sig)
    py = prior_ln(y, lo, hi)
    ly = np.full(Wn, -np.inf)
    inside = np.isfinite(py)
    if inside.any():
        ly[inside] = target(y[inside])
    lr = np.where(beta > 0.0, beta * (ly - lnl), 0.0) + (py - lnp) + (qx - qy)
    acc = inside & (np.log(accept_units(seed, step, range(Wn))) < lr)
    x2, l2, p2 = x.copy(), lnl.copy(), lnp.copy()
    x2[acc], l2[acc], p2[acc] = y[acc], ly[acc], py[acc]
    return x2, l2, p2, acc, lr


def minibatch_index(seed):
    """Minibatch rows of training round r, iteration i: Philox counters (r, 5, i, j / 4),
    word j mod 4, scaled to [0, n)."""
    def fn(i, batch, n, rnd=0):
        out = np.empty(batch, dtype=np.int64)
        for q in range(0, batch, 4):
            u = _philox_units(seed, (rnd, 5, i, q // 4))
            for k in range(min(4, batch - q)):
                out[q + k] = min(int(u[k] * n), n - 1)
        return out
    return fn
