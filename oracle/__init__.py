"""Plain FP64 CPU oracle for the batched LISA log-likelihood (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` may import this package.  The product library never loads it
and shares no code with it.  The arithmetic lives in ``lisa_oracle.c`` (plain C,
FP64, ``-ffp-contract=off``); this module compiles it with gcc and wraps it with
ctypes and numpy.

Every function follows a passage of Katz et al. (2020), Sec. II and II.A: the
mode model of Eq. (5), the time-frequency map of Eq. (6), the response of
Eqs. (7)-(10), the sparse-knot cubic splines, and the likelihood of Eqs. (2),
(3) and (11).  Stand-in coefficients are flagged STANDIN in the C source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lisa_oracle.c")
_SRCS = (_SRC, os.path.join(_HERE, "oracle_sampler.c"))
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODES6 = ((2, 2), (3, 3), (4, 4), (2, 1), (3, 2), (4, 3))
NPAR = 11
NSERIES = 8


def build(force: bool = False) -> str:
    """Compile lisa_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    deps = _SRCS + (os.path.join(_HERE, "oracle.h"),)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(p) for p in deps
    ):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, *_SRCS, "-lm"]
    subprocess.check_call(cmd, cwd=_HERE)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            lp = C.POINTER(C.c_int64)
            i64 = C.c_int64
            d = C.c_double
            i = C.c_int
            L.oracle_sylm.argtypes = [i, i, i, d, d, dp, dp]
            L.oracle_sylm.restype = None
            L.oracle_mode_eval.argtypes = [dp, d, i, i, dp, i64, dp, dp, dp, dp]
            L.oracle_peak_and_cut.argtypes = [dp, i, i, dp, dp]
            L.oracle_orbit.argtypes = [d, dp, dp]
            L.oracle_orbit.restype = None
            L.oracle_transfer.argtypes = [dp, i, i, dp, dp, i64, dp]
            L.oracle_delay_phase.argtypes = [dp, d, d]
            L.oracle_delay_phase.restype = d
            L.oracle_band.argtypes = [dp, d, i, i, d, d, i64, dp, dp, lp, lp]
            L.oracle_knots.argtypes = [dp, d, i, i, d, d, i64, i, dp, dp]
            L.oracle_spline.argtypes = [i, dp, dp, dp]
            L.oracle_spline_eval.argtypes = [i, dp, dp, dp, i64, dp]
            L.oracle_spline_eval.restype = None
            L.oracle_template.argtypes = [dp, d, ip, i, i, d, d, i64, dp]
            L.oracle_direct.argtypes = [dp, d, ip, i, d, d, i64, dp]
            L.oracle_mode_response.argtypes = [dp, d, i, i, d, d, i64, dp, i64, dp]
            L.oracle_inner.argtypes = [dp, dp, dp, d, i64]
            L.oracle_inner.restype = d
            L.oracle_loglike.argtypes = [dp, i, d, ip, i, i, d, d, i64, dp, dp, i, dp, dp, dp, dp]
            L.oracle_loglike_residual.argtypes = [dp, d, ip, i, i, d, d, i64, dp, dp, dp]
            L.oracle_psd_aet.argtypes = [dp, i64, dp]
            L.oracle_psd_aet.restype = None
            L.oracle_noise.argtypes = [dp, d, i64, dp, dp]
            L.oracle_noise.restype = None
            L.oracle_dl_gpc.argtypes = [d]
            L.oracle_dl_gpc.restype = d
            L.oracle_polarizations.argtypes = [dp, d, i, i, dp, i64, dp, dp]
            u32p = C.POINTER(C.c_uint32)
            llp = C.POINTER(C.c_longlong)
            cfgp = C.POINTER(SamplerCfg)
            L.oracle_philox.argtypes = [u32p, u32p, u32p]
            L.oracle_philox.restype = None
            for fn in (L.oracle_lisa_to_ssb, L.oracle_ssb_to_lisa):
                fn.argtypes = [dp, dp]
                fn.restype = None
            L.oracle_to_physical.argtypes = [dp, i, d, dp]
            L.oracle_to_physical.restype = None
            L.oracle_default_ladder.argtypes = [i, d, i, dp]
            L.oracle_default_ladder.restype = None
            L.oracle_adapt_ladder.argtypes = [i, dp, dp, d]
            L.oracle_adapt_ladder.restype = None
            L.oracle_sampler_gauss.argtypes = [cfgp, dp, dp, i, i, dp, dp, dp, dp, llp, llp]
            L.oracle_sampler_lisa.argtypes = [cfgp, d, ip, i, i, d, d, i64, dp, dp, i, i, i, dp,
                                              dp, dp, dp, llp, llp]
            L.oracle_autocorr_time.argtypes = [dp, i, i, dp]
            L.oracle_autocorr_time.restype = d
            _lib = L
    return _lib


class SamplerCfg(C.Structure):
    """Mirror of oracle_sampler_cfg."""
    _fields_ = [("T", C.c_int), ("W", C.c_int), ("a", C.c_double),
                ("betas", C.POINTER(C.c_double)), ("adaptive", C.c_int),
                ("adapt_lag", C.c_double), ("adapt_time", C.c_double),
                ("seed", C.c_uint64), ("lower", C.POINTER(C.c_double)),
                ("upper", C.POINTER(C.c_double)), ("lisa_frame", C.c_int)]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _modes(modes):
    return np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1, 2))


# --------------------------------------------------------------------------- pieces

def sylm(s: int, l: int, m: int, theta: float, phi: float) -> complex:
    """Spin-weighted spherical harmonic sY_lm (Goldberg closed form)."""
    re, im = C.c_double(), C.c_double()
    lib().oracle_sylm(s, l, m, theta, phi, C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def mode_eval(th, t0, l, m, f):
    """Amplitude, phase, dphase/df and t_lm(f) of mode (l,m) (Eqs. (5), (6))."""
    th, f = _f64(th), _f64(f)
    n = f.size
    a, p, dp_, t = (np.empty(n) for _ in range(4))
    ok = lib().oracle_mode_eval(_dp(th), t0, l, m, _dp(f), n, _dp(a), _dp(p), _dp(dp_), _dp(t))
    if not ok:
        raise ValueError("invalid parameters or mode")
    return a, p, dp_, t


def peak_and_cut(th, l=2, m=2):
    fp, fc = C.c_double(), C.c_double()
    if not lib().oracle_peak_and_cut(_dp(_f64(th)), l, m, C.byref(fp), C.byref(fc)):
        raise ValueError("invalid parameters or mode")
    return fp.value, fc.value


def orbit(t):
    p0, q = np.empty(3), np.empty(9)
    lib().oracle_orbit(float(t), _dp(p0), _dp(q))
    return p0, q.reshape(3, 3)


def transfer(th, l, m, f, t):
    th, f, t = _f64(th), _f64(f), _f64(t)
    n = f.size
    T = np.empty((3, n, 2))
    if not lib().oracle_transfer(_dp(th), l, m, _dp(f), _dp(t), n, _dp(T)):
        raise ValueError("invalid parameters or mode")
    return T[..., 0] + 1j * T[..., 1]


def delay_phase(th, f, t):
    return lib().oracle_delay_phase(_dp(_f64(th)), float(f), float(t))


def band(th, t0, l, m, f0, df, n_bins):
    flo, fhi = C.c_double(), C.c_double()
    jlo, jhi = C.c_int64(), C.c_int64()
    ok = lib().oracle_band(_dp(_f64(th)), t0, l, m, f0, df, n_bins, C.byref(flo), C.byref(fhi),
                           C.byref(jlo), C.byref(jhi))
    if not ok:
        return None
    return flo.value, fhi.value, jlo.value, jhi.value


def knots(th, t0, l, m, f0, df, n_bins, K):
    fk = np.empty(K)
    vals = np.empty((NSERIES, K))
    ok = lib().oracle_knots(_dp(_f64(th)), t0, l, m, f0, df, n_bins, K, _dp(fk), _dp(vals))
    if not ok:
        return None
    return fk, vals


def spline(x, y):
    x, y = _f64(x), _f64(y)
    K = x.size
    c = np.empty((K - 1, 4))
    if not lib().oracle_spline(K, _dp(x), _dp(y), _dp(c)):
        raise ValueError("need at least 4 knots")
    return c


def spline_eval(xk, c, f):
    xk, c, f = _f64(xk), _f64(c), _f64(f)
    y = np.empty(f.size)
    lib().oracle_spline_eval(xk.size, _dp(xk), _dp(c), _dp(f), f.size, _dp(y))
    return y


def template(th, t0, modes, K, f0, df, n_bins):
    """Dense template h[3, n_bins] (complex) by knots -> splines -> bins."""
    md = _modes(modes)
    h = np.empty((3, n_bins, 2))
    lib().oracle_template(_dp(_f64(th)), t0, md.ctypes.data_as(C.POINTER(C.c_int)), len(md), K,
                          f0, df, n_bins, _dp(h))
    return h[..., 0] + 1j * h[..., 1]


def direct(th, t0, modes, f0, df, n_bins):
    """Dense template by direct waveform + response evaluation at every bin."""
    md = _modes(modes)
    h = np.empty((3, n_bins, 2))
    lib().oracle_direct(_dp(_f64(th)), t0, md.ctypes.data_as(C.POINTER(C.c_int)), len(md), f0,
                        df, n_bins, _dp(h))
    return h[..., 0] + 1j * h[..., 1]


def mode_response(th, t0, l, m, f0, df, n_bins, f):
    """One mode's A, E, T response [3, n] (complex) at arbitrary frequencies f (direct
    evaluation; zero outside the mode's band on the grid)."""
    f = _f64(f)
    h = np.empty((3, f.size, 2))
    if not lib().oracle_mode_response(_dp(_f64(th)), t0, l, m, f0, df, n_bins, _dp(f), f.size,
                                      _dp(h)):
        raise ValueError("invalid parameters or mode")
    return h[..., 0] + 1j * h[..., 1]


def _cplx_pairs(a):
    a = np.asarray(a)
    if np.iscomplexobj(a):
        return _f64(np.stack([a.real, a.imag], axis=-1))
    return _f64(a)


def inner(a, b, psd, df):
    a2, b2, p = _cplx_pairs(a), _cplx_pairs(b), _f64(psd)
    n = p.shape[-1]
    return lib().oracle_inner(_dp(a2), _dp(b2), _dp(p), df, n)


def loglike(th, t0, modes, K, f0, df, d, psd, n_threads=None):
    """Batched ln L (Eq. (2)); returns lnL, <d|h>, <h|h>, <d|d>."""
    th = _f64(np.atleast_2d(th))
    B = th.shape[0]
    md = _modes(modes)
    d2, p = _cplx_pairs(d), _f64(psd)
    n_bins = p.shape[-1]
    lnL, dh, hh = np.empty(B), np.empty(B), np.empty(B)
    dd = C.c_double()
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    ok = lib().oracle_loglike(_dp(th), B, t0, md.ctypes.data_as(C.POINTER(C.c_int)), len(md), K,
                              f0, df, n_bins, _dp(d2), _dp(p), int(n_threads), _dp(lnL), _dp(dh),
                              _dp(hh), C.byref(dd))
    if not ok:
        raise ValueError("invalid arguments")
    return lnL, dh, hh, dd.value


def loglike_residual(th, t0, modes, K, f0, df, d, psd):
    md = _modes(modes)
    d2, p = _cplx_pairs(d), _f64(psd)
    out = C.c_double()
    ok = lib().oracle_loglike_residual(_dp(_f64(th)), t0, md.ctypes.data_as(C.POINTER(C.c_int)),
                                       len(md), K, f0, df, p.shape[-1], _dp(d2), _dp(p),
                                       C.byref(out))
    if not ok:
        raise ValueError("invalid arguments")
    return out.value


def psd_aet(f):
    f = _f64(f)
    S = np.empty((3, f.size))
    lib().oracle_psd_aet(_dp(f), f.size, _dp(S))
    return S


def noise(psd, df, z):
    """Coloured noise of Eq. (12) from white normal pairs z[3, n, 2]."""
    p, z = _f64(psd), _f64(z)
    n_bins = p.shape[-1]
    out = np.empty((3, n_bins, 2))
    lib().oracle_noise(_dp(p), df, n_bins, _dp(z), _dp(out))
    return out[..., 0] + 1j * out[..., 1]


def dl_gpc(z):
    return lib().oracle_dl_gpc(float(z))


def polarizations(th, t0, l, m, f):
    f = _f64(f)
    hp, hc = np.empty((f.size, 2)), np.empty((f.size, 2))
    if not lib().oracle_polarizations(_dp(_f64(th)), t0, l, m, _dp(f), f.size, _dp(hp), _dp(hc)):
        raise ValueError("invalid parameters or mode")
    return hp[:, 0] + 1j * hp[:, 1], hc[:, 0] + 1j * hc[:, 1]


# --------------------------------------------------------------------------- sampler

def philox(ctr, key):
    """One Philox4x32-10 block (Salmon et al. 2011): four uint32 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.empty(4, dtype=np.uint32)
    u32p = C.POINTER(C.c_uint32)
    lib().oracle_philox(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), o.ctypes.data_as(u32p))
    return o


def lisa_to_ssb(t, lam, beta, psi):
    """LISA frame -> SSB frame: (t_L, lambda_L, beta_L, psi_L) -> (t, lambda, beta, psi)."""
    o = np.empty(4)
    lib().oracle_lisa_to_ssb(_dp(_f64([t, lam, beta, psi])), _dp(o))
    return tuple(o)


def ssb_to_lisa(t, lam, beta, psi):
    o = np.empty(4)
    lib().oracle_ssb_to_lisa(_dp(_f64([t, lam, beta, psi])), _dp(o))
    return tuple(o)


def from_physical(th):
    """Sampling coordinates of Table I from physical parameters (SSB frame)."""
    th = _f64(th)
    return np.array([np.log(th[0]), th[1], th[2], th[3], np.log(th[4]), th[5], np.cos(th[6]),
                     th[7], np.sin(th[8]), th[9], np.log(th[10])])


def to_physical(x, lisa_frame=False, t0=0.0):
    """Physical parameters from the sampling coordinates of Table I."""
    x = _f64(x)
    th = np.empty(NPAR)
    lib().oracle_to_physical(_dp(x), int(lisa_frame), float(t0), _dp(th))
    return th


def default_ladder(T, ratio=2.04807, t_max_inf=True):
    b = np.empty(T)
    lib().oracle_default_ladder(int(T), float(ratio), int(t_max_inf), _dp(b))
    return b


def adapt_ladder(betas, A, kappa):
    b = _f64(betas).copy()
    lib().oracle_adapt_ladder(b.size, _dp(b), _dp(_f64(A)), float(kappa))
    return b


class SamplerRun:
    """Result of an oracle sampler run: final state, cold chain, counters, ladder."""

    def __init__(self, x, lnl, chain, lnl_chain, acc, swaps, betas):
        self.x, self.lnl, self.chain, self.lnl_chain = x, lnl, chain, lnl_chain
        self.acc, self.swaps, self.betas = acc, swaps, betas


def _sampler_cfg(x, betas, a, seed, lower, upper, adaptive, adapt_lag, adapt_time, lisa_frame):
    T, W = x.shape[0], x.shape[1]
    keep = dict(betas=_f64(betas).copy(), lo=_f64(lower), hi=_f64(upper))
    cfg = SamplerCfg(T=T, W=W, a=float(a), betas=_dp(keep["betas"]), adaptive=int(adaptive),
                     adapt_lag=float(adapt_lag), adapt_time=float(adapt_time), seed=int(seed),
                     lower=_dp(keep["lo"]), upper=_dp(keep["hi"]), lisa_frame=int(lisa_frame))
    return cfg, keep


def _sampler_out(T, W, n_steps):
    return (np.empty((n_steps, W, NPAR)), np.empty((n_steps, W)), np.zeros((T, 2), np.int64),
            np.zeros((T, 2), np.int64), np.empty((T, W)))


def sampler_gauss(x0, betas, mean, sigma, n_steps, seed, lower, upper, a=1.15, step0=0,
                  adaptive=False, adapt_lag=10000.0, adapt_time=100.0):
    """PT stretch sampler (Sec. III) on N(mean, diag(sigma^2)); x0 [T, W, 11]."""
    x = _f64(x0).copy()
    T, W = x.shape[0], x.shape[1]
    cfg, keep = _sampler_cfg(x, betas, a, seed, lower, upper, adaptive, adapt_lag, adapt_time,
                             False)
    chain, lch, acc, sw, lnl = _sampler_out(T, W, n_steps)
    llp = C.POINTER(C.c_longlong)
    ok = lib().oracle_sampler_gauss(C.byref(cfg), _dp(_f64(mean)), _dp(_f64(sigma)), int(step0),
                                    int(n_steps), _dp(x), _dp(lnl), _dp(chain), _dp(lch),
                                    acc.ctypes.data_as(llp), sw.ctypes.data_as(llp))
    if not ok:
        raise ValueError("invalid sampler arguments")
    return SamplerRun(x, lnl, chain, lch, acc, sw, keep["betas"])


def sampler_lisa(x0, betas, n_steps, seed, lower, upper, t0, modes, K, f0, df, d, psd,
                 a=1.15, step0=0, adaptive=False, adapt_lag=10000.0, adapt_time=100.0,
                 lisa_frame=True, n_threads=None):
    """PT stretch sampler (Sec. III) on the LISA likelihood of Eq. (2)."""
    x = _f64(x0).copy()
    T, W = x.shape[0], x.shape[1]
    cfg, keep = _sampler_cfg(x, betas, a, seed, lower, upper, adaptive, adapt_lag, adapt_time,
                             lisa_frame)
    chain, lch, acc, sw, lnl = _sampler_out(T, W, n_steps)
    md = _modes(modes)
    d2, p = _cplx_pairs(d), _f64(psd)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    llp = C.POINTER(C.c_longlong)
    ok = lib().oracle_sampler_lisa(C.byref(cfg), float(t0), md.ctypes.data_as(C.POINTER(C.c_int)),
                                   len(md), int(K), float(f0), float(df), p.shape[-1], _dp(d2),
                                   _dp(p), int(n_threads), int(step0), int(n_steps), _dp(x),
                                   _dp(lnl), _dp(chain), _dp(lch), acc.ctypes.data_as(llp),
                                   sw.ctypes.data_as(llp))
    if not ok:
        raise ValueError("invalid sampler arguments")
    return SamplerRun(x, lnl, chain, lch, acc, sw, keep["betas"])


def autocorr_time(series, return_rho=False):
    """Sec. III.C estimator on series[n, W] (one parameter, every walker)."""
    s = _f64(series)
    n, W = s.shape
    rho = np.empty(n)
    tau = lib().oracle_autocorr_time(_dp(s), n, W, _dp(rho))
    return (tau, rho) if return_rho else tau
