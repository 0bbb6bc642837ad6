"""ctypes binding of liblisalike.so (include/lisa_like.h), argument marshalling only.

Function names match the C ABI.  Every step of the likelihood runs in the CUDA
library; this module converts numpy arrays / torch tensors to pointers and checks
status codes.  Loading fails loudly when the library is missing: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblisalike.so")

LISA_OK, LISA_ERR_ARG, LISA_ERR_STATE, LISA_ERR_CUDA, LISA_ERR_OOM, LISA_ERR_TIMEOUT = range(6)
LISA_PREC_FP64, LISA_PREC_SPLIT = 0, 1
STATUS_NAMES = {0: "LISA_OK", 1: "LISA_ERR_ARG", 2: "LISA_ERR_STATE", 3: "LISA_ERR_CUDA",
                4: "LISA_ERR_OOM", 5: "LISA_ERR_TIMEOUT"}
MODES6 = ((2, 2), (3, 3), (4, 4), (2, 1), (3, 2), (4, 3))
NPAR = 11

# exported symbols (the set the header declares)
SYMBOLS = (
    "lisa_like_default_config", "lisa_like_create", "lisa_like_set_data", "lisa_like_loglike",
    "lisa_like_loglike_device", "lisa_like_data_inner", "lisa_like_template",
    "lisa_like_stage_knots", "lisa_like_stage_coeffs", "lisa_dl_from_z", "lisa_psd_aet",
    "lisa_like_last_launches", "lisa_like_destroy", "lisa_like_last_error",
    "lisa_like_set_profiling", "lisa_like_read_profile", "lisa_like_loglike_noalloc",
    "lisa_like_set_graphs", "lisa_like_test_device_wait", "lisa_like_set_tune", "lisa_like_get_tune", "lisa_like_autotune",
    "lisa_like_mode_inner", "lisa_like_mode_cross", "lisa_like_set_fiducial", "lisa_like_rb_edges",
    "lisa_like_loglike_rb", "lisa_like_loglike_rb_device",
    # include/lisa_sampler.h
    "lisa_sampler_default_config", "lisa_sampler_create", "lisa_sampler_set_ladder",
    "lisa_sampler_set_state", "lisa_sampler_run", "lisa_sampler_get_state",
    "lisa_sampler_get_counts", "lisa_sampler_step_launches", "lisa_sampler_destroy",
    "lisa_sampler_last_error", "lisa_sampler_to_physical", "lisa_sampler_from_physical",
    "lisa_sampler_sky_mode_init",
    "lisa_autocorr_time", "lisa_flow_default_schedule", "lisa_sampler_enable_flow",
    "lisa_sampler_get_flow", "lisa_sampler_flow_stats", "lisa_sampler_set_flow_likelihood",
    "lisa_sampler_set_flow_screen", "lisa_sampler_flow_screen_count",
    # include/lisa_probe.h
    "lisa_probe_pipes",
    # include/lisa_flow.h
    "lisa_flow_create", "lisa_flow_destroy", "lisa_flow_last_error", "lisa_flow_set_weights",
    "lisa_flow_get_weights", "lisa_flow_set_whitening", "lisa_flow_get_whitening",
    "lisa_flow_normalize", "lisa_flow_generate", "lisa_flow_gradients", "lisa_flow_train",
)
FLOW_COUPLINGS, FLOW_HIDDEN, FLOW_PARAMS_PER_COUPLING = 8, 128, 20886
LISA_TARGET_LIKELIHOOD, LISA_TARGET_GAUSSIAN = 0, 1
SAMPLER_NDIM = 11
NOALLOC_SCRATCH_BYTES = 4194304
NOALLOC_MAX_WALKER_MODE_KNOTS = 8192
NOALLOC_MAX_ITEMS = 16384


class lisa_like_config(C.Structure):
    _fields_ = [
        ("n_modes", C.c_int),
        ("modes", (C.c_int * 2) * 6),
        ("n_knots", C.c_int),
        ("precision", C.c_int),
        ("t0_s", C.c_double),
        ("device", C.c_int),
        ("stream", C.c_void_p),
        ("max_batch", C.c_int),
        ("timeout_s", C.c_double),
    ]


class lisa_sampler_config(C.Structure):
    _fields_ = [
        ("n_temps", C.c_int),
        ("n_walkers", C.c_int),
        ("a", C.c_double),
        ("ladder_ratio", C.c_double),
        ("t_max_inf", C.c_int),
        ("adaptive", C.c_int),
        ("adapt_lag", C.c_double),
        ("adapt_time", C.c_double),
        ("seed", C.c_uint64),
        ("lower", C.c_double * 11),
        ("upper", C.c_double * 11),
        ("lisa_frame", C.c_int),
        ("target", C.c_int),
        ("gauss_mean", C.c_double * 11),
        ("gauss_sigma", C.c_double * 11),
        ("use_graphs", C.c_int),
        ("timeout_s", C.c_double),
    ]


class lisa_flow_schedule(C.Structure):
    _fields_ = [
        ("train_every", C.c_int),
        ("train_iters", C.c_int),
        ("batch", C.c_int),
        ("lr", C.c_double),
        ("freeze_after", C.c_int),
        ("seed", C.c_uint64),
        ("flow_only", C.c_int),
    ]


class LisaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load liblisalike.so (build it first with paper_2005_01827_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("liblisalike.so not found at %s; build it with "
                          "`python -m paper_2005_01827_gb300.build`" % path)
    L = C.CDLL(path)
    vp, dp, i, i64, d = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_int64, C.c_double
    cfgp = C.POINTER(lisa_like_config)
    L.lisa_like_default_config.argtypes = [cfgp]
    L.lisa_like_default_config.restype = None
    L.lisa_like_create.argtypes = [cfgp, C.POINTER(vp)]
    L.lisa_like_create.restype = i
    L.lisa_like_set_data.argtypes = [vp, d, d, i64, vp, vp]
    L.lisa_like_set_data.restype = i
    L.lisa_like_loglike.argtypes = [vp, vp, i, vp, vp, vp]
    L.lisa_like_loglike.restype = i
    L.lisa_like_loglike_device.argtypes = [vp, vp, i, vp, vp, vp, vp]
    L.lisa_like_loglike_device.restype = i
    L.lisa_like_data_inner.argtypes = [vp, dp]
    L.lisa_like_data_inner.restype = i
    L.lisa_like_template.argtypes = [vp, vp, vp]
    L.lisa_like_template.restype = i
    L.lisa_like_stage_knots.argtypes = [vp, vp, i, vp, vp, vp, vp]
    L.lisa_like_stage_knots.restype = i
    L.lisa_like_stage_coeffs.argtypes = [vp, vp, i, vp]
    L.lisa_like_stage_coeffs.restype = i
    L.lisa_dl_from_z.argtypes = [d]
    L.lisa_dl_from_z.restype = d
    L.lisa_psd_aet.argtypes = [d, d, i64, vp]
    L.lisa_psd_aet.restype = i
    L.lisa_like_set_profiling.argtypes = [vp, i]
    L.lisa_like_set_profiling.restype = i
    L.lisa_like_read_profile.argtypes = [vp, dp, C.POINTER(C.c_int)]
    L.lisa_like_read_profile.restype = i
    L.lisa_like_loglike_noalloc.argtypes = [cfgp, d, d, i64, vp, d, vp, i, vp, vp, vp, vp]
    L.lisa_like_loglike_noalloc.restype = i
    ip = C.POINTER(C.c_int)
    L.lisa_like_set_graphs.argtypes = [vp, i]
    L.lisa_like_set_graphs.restype = i
    L.lisa_like_test_device_wait.argtypes = [vp, i]
    L.lisa_like_test_device_wait.restype = i
    L.lisa_like_set_tune.argtypes = [vp, i, i]
    L.lisa_like_set_tune.restype = i
    L.lisa_like_get_tune.argtypes = [vp, ip]
    L.lisa_like_get_tune.restype = i
    L.lisa_like_autotune.argtypes = [vp, vp, i, ip]
    L.lisa_like_autotune.restype = i
    L.lisa_like_mode_inner.argtypes = [vp, vp, i, vp, vp]
    L.lisa_like_mode_inner.restype = i
    L.lisa_like_mode_cross.argtypes = [vp, vp, i, vp]
    L.lisa_like_mode_cross.restype = i
    L.lisa_like_set_fiducial.argtypes = [vp, vp, i]
    L.lisa_like_rb_edges.argtypes = [vp, vp, ip]
    L.lisa_like_loglike_rb.argtypes = [vp, vp, i, vp, vp, vp]
    L.lisa_like_loglike_rb_device.argtypes = [vp, vp, i, vp, vp, vp, vp]
    for fn in ("lisa_like_set_fiducial", "lisa_like_rb_edges", "lisa_like_loglike_rb",
               "lisa_like_loglike_rb_device"):
        getattr(L, fn).restype = i
    L.lisa_like_last_launches.argtypes = [vp]
    L.lisa_like_last_launches.restype = i
    L.lisa_like_destroy.argtypes = [vp]
    L.lisa_like_destroy.restype = None
    L.lisa_like_last_error.argtypes = [vp]
    L.lisa_like_last_error.restype = C.c_char_p
    scfgp = C.POINTER(lisa_sampler_config)
    u32, u64 = C.c_uint32, C.c_uint64
    L.lisa_sampler_default_config.argtypes = [scfgp]
    L.lisa_sampler_default_config.restype = None
    L.lisa_sampler_create.argtypes = [vp, scfgp, C.POINTER(vp)]
    L.lisa_sampler_set_ladder.argtypes = [vp, vp]
    L.lisa_sampler_set_state.argtypes = [vp, vp, u32]
    L.lisa_sampler_run.argtypes = [vp, i, vp, vp]
    L.lisa_sampler_get_state.argtypes = [vp, vp, vp, vp, C.POINTER(u32)]
    L.lisa_sampler_get_counts.argtypes = [vp, vp, vp]
    L.lisa_sampler_step_launches.argtypes = [vp]
    L.lisa_sampler_destroy.argtypes = [vp]
    L.lisa_sampler_destroy.restype = None
    L.lisa_sampler_last_error.argtypes = [vp]
    L.lisa_sampler_last_error.restype = C.c_char_p
    L.lisa_sampler_to_physical.argtypes = [vp, i, i, d, vp, vp]
    L.lisa_sampler_from_physical.argtypes = [vp, i, i, d, vp]
    L.lisa_sampler_sky_mode_init.argtypes = [vp, vp, vp, vp, i, i, u64, vp]
    L.lisa_autocorr_time.argtypes = [vp, i, i, i, i, dp, vp, vp]
    L.lisa_probe_pipes.argtypes = [i, dp]
    L.lisa_probe_pipes.restype = i
    fsp = C.POINTER(lisa_flow_schedule)
    L.lisa_flow_default_schedule.argtypes = [fsp]
    L.lisa_flow_default_schedule.restype = None
    L.lisa_sampler_enable_flow.argtypes = [vp, fsp]
    L.lisa_sampler_get_flow.argtypes = [vp]
    L.lisa_sampler_get_flow.restype = vp
    L.lisa_sampler_flow_stats.argtypes = [vp, vp, C.POINTER(C.c_int), dp]
    L.lisa_sampler_set_flow_likelihood.argtypes = [vp, vp]
    L.lisa_sampler_set_flow_likelihood.restype = i
    L.lisa_sampler_set_flow_screen.argtypes = [vp, d]
    L.lisa_sampler_set_flow_screen.restype = i
    L.lisa_sampler_flow_screen_count.argtypes = [vp, C.POINTER(C.c_int64)]
    L.lisa_sampler_flow_screen_count.restype = i
    L.lisa_flow_create.argtypes = [u64, C.POINTER(vp)]
    L.lisa_flow_destroy.argtypes = [vp]
    L.lisa_flow_destroy.restype = None
    L.lisa_flow_last_error.argtypes = [vp]
    L.lisa_flow_last_error.restype = C.c_char_p
    L.lisa_flow_set_weights.argtypes = [vp, vp]
    L.lisa_flow_get_weights.argtypes = [vp, vp]
    L.lisa_flow_set_whitening.argtypes = [vp, vp, vp]
    L.lisa_flow_get_whitening.argtypes = [vp, vp, vp]
    L.lisa_flow_normalize.argtypes = [vp, vp, i, vp, vp, vp]
    L.lisa_flow_generate.argtypes = [vp, vp, i, vp, vp, vp]
    L.lisa_flow_gradients.argtypes = [vp, vp, i, vp, dp, vp]
    L.lisa_flow_train.argtypes = [vp, vp, i64, i, i, d, u64, u32, vp, vp]
    for fn in ("lisa_sampler_enable_flow", "lisa_sampler_flow_stats", "lisa_flow_create",
               "lisa_flow_set_weights", "lisa_flow_get_weights", "lisa_flow_set_whitening",
               "lisa_flow_get_whitening", "lisa_flow_normalize", "lisa_flow_generate",
               "lisa_flow_gradients", "lisa_flow_train"):
        getattr(L, fn).restype = i
    for fn in ("lisa_sampler_create", "lisa_sampler_set_ladder", "lisa_sampler_set_state",
               "lisa_sampler_run", "lisa_sampler_get_state", "lisa_sampler_get_counts",
               "lisa_sampler_step_launches", "lisa_sampler_to_physical",
               "lisa_sampler_sky_mode_init", "lisa_autocorr_time", "lisa_sampler_from_physical"):
        getattr(L, fn).restype = i
    _lib = L
    return L


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):            # torch tensor (host or device)
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _require_device_f64(t, n, name):
    """A tensor handed to an entry point that takes raw device addresses must be a
    contiguous float64 CUDA tensor of at least n elements (None passes)."""
    if t is None or not hasattr(t, "data_ptr"):
        return
    if str(t.dtype) != "torch.float64" or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} elements, the call needs {n}")


def _check(st, h=None):
    if st != LISA_OK:
        raise LisaError(st, lisa_like_last_error(h))


# ------------------------------------------------------------------- C-named wrappers

def lisa_like_default_config() -> lisa_like_config:
    cfg = lisa_like_config()
    load().lisa_like_default_config(C.byref(cfg))
    return cfg


def lisa_like_create(cfg: lisa_like_config):
    h = C.c_void_p()
    _check(load().lisa_like_create(C.byref(cfg), C.byref(h)))
    return h


def lisa_like_set_data(h, f0, df, n_bins, d, psd):
    d = None if d is None else _f64(d)
    psd = _f64(psd)
    _check(load().lisa_like_set_data(h, f0, df, n_bins, _ptr(d), _ptr(psd)), h)


def lisa_like_loglike(h, params, B, lnL, dh=None, hh=None):
    _check(load().lisa_like_loglike(h, _ptr(params), B, _ptr(lnL), _ptr(dh), _ptr(hh)), h)


def lisa_like_loglike_device(h, d_params, B, d_lnL, d_dh=None, d_hh=None, stream=None):
    s = None if stream is None else C.c_void_p(int(stream))
    _check(load().lisa_like_loglike_device(h, _ptr(d_params), B, _ptr(d_lnL), _ptr(d_dh),
                                           _ptr(d_hh), s), h)


def lisa_like_loglike_rb_device(h, d_params, B, d_lnL, d_dh=None, d_hh=None, stream=None):
    s = None if stream is None else C.c_void_p(int(stream))
    _check(load().lisa_like_loglike_rb_device(h, _ptr(d_params), B, _ptr(d_lnL), _ptr(d_dh),
                                              _ptr(d_hh), s), h)


def lisa_like_data_inner(h) -> float:
    v = C.c_double()
    _check(load().lisa_like_data_inner(h, C.byref(v)), h)
    return v.value


def lisa_like_template(h, params, out):
    _check(load().lisa_like_template(h, _ptr(params), _ptr(out)), h)


def lisa_like_stage_knots(h, params, B, band=None, fedge=None, fk=None, vals=None):
    _check(load().lisa_like_stage_knots(h, _ptr(params), B, _ptr(band), _ptr(fedge), _ptr(fk),
                                        _ptr(vals)), h)


def lisa_like_stage_coeffs(h, params, B, coef):
    _check(load().lisa_like_stage_coeffs(h, _ptr(params), B, _ptr(coef)), h)


def lisa_dl_from_z(z: float) -> float:
    return load().lisa_dl_from_z(float(z))


def lisa_psd_aet(f0, df, n_bins, out):
    _check(load().lisa_psd_aet(f0, df, n_bins, _ptr(out)))


def lisa_like_set_profiling(h, on: bool):
    _check(load().lisa_like_set_profiling(h, int(bool(on))), h)


def lisa_like_read_profile(h):
    """Per-stage device ms summed since the last read: knots, splines, segment prep,
    plan, dense, finish; and the number of calls."""
    ms = (C.c_double * 6)()
    n = C.c_int()
    _check(load().lisa_like_read_profile(h, ms, C.byref(n)), h)
    return list(ms), n.value


def lisa_like_loglike_noalloc(cfg, f0, df, n_bins, d_bins, dd, d_params, B, d_lnL, d_dh=None,
                              d_hh=None, stream=None):
    """Allocation-free batched ln L on caller-owned device buffers (see the header).

    Tensor arguments must be contiguous float64 CUDA tensors at least as large as the
    call reads or writes: the C entry point only sees their addresses."""
    for t, need, name in ((d_bins, 9 * int(n_bins), "d_bins"), (d_params, 11 * int(B), "d_params"),
                          (d_lnL, int(B), "d_lnL"), (d_dh, int(B), "d_dh"), (d_hh, int(B), "d_hh")):
        _require_device_f64(t, need, name)
    s = None if stream is None else C.c_void_p(int(stream))
    _check(load().lisa_like_loglike_noalloc(C.byref(cfg), f0, df, n_bins, _ptr(d_bins), dd,
                                            _ptr(d_params), B, _ptr(d_lnL), _ptr(d_dh),
                                            _ptr(d_hh), s))


def lisa_like_set_graphs(h, on: bool):
    _check(load().lisa_like_set_graphs(h, int(bool(on))), h)


def lisa_like_test_device_wait(h, polls: int):
    """Test of the device-side timeout path: later calls arm the staging barrier without
    a copy and give up after `polls` polls (0 = normal operation)."""
    _check(load().lisa_like_test_device_wait(h, int(polls)), h)


def lisa_like_set_tune(h, per_thread: int, group: int):
    _check(load().lisa_like_set_tune(h, per_thread, group), h)


def lisa_like_get_tune(h):
    out = (C.c_int * 3)()
    _check(load().lisa_like_get_tune(h, out), h)
    return tuple(out)


def lisa_like_autotune(h, params, B):
    """Time the supported dense tile shapes on these walkers and keep the fastest."""
    out = (C.c_int * 3)()
    p = _f64(params)
    _check(load().lisa_like_autotune(h, _ptr(p), B, out), h)
    return tuple(out)


def lisa_like_mode_inner(h, params, B, dh_modes=None, hh_modes=None):
    _check(load().lisa_like_mode_inner(h, _ptr(params), B, _ptr(dh_modes), _ptr(hh_modes)), h)


def lisa_like_last_launches(h) -> int:
    return load().lisa_like_last_launches(h)


def lisa_like_destroy(h):
    load().lisa_like_destroy(h)


def lisa_like_last_error(h=None) -> str:
    msg = load().lisa_like_last_error(h)
    return msg.decode() if msg else ""


# ------------------------------------------------------------------- convenience class

class LisaLike:
    """Owns one handle.  Arrays are numpy (host) unless a method says device."""

    def __init__(self, modes=MODES6, n_knots=1024, precision=LISA_PREC_FP64, t0=3.15576e7,
                 max_batch=1024, device=0, stream=None, timeout_s=60.0):
        cfg = lisa_like_default_config()
        cfg.n_modes = len(modes)
        for k, (l, m) in enumerate(modes):
            cfg.modes[k][0], cfg.modes[k][1] = l, m
        cfg.n_knots, cfg.precision, cfg.t0_s = n_knots, precision, t0
        cfg.max_batch, cfg.device, cfg.timeout_s = max_batch, device, timeout_s
        cfg.stream = None if stream is None else int(stream)
        self.modes, self.K, self.L = tuple(modes), n_knots, len(modes)
        self.max_batch = max_batch
        self.h = lisa_like_create(cfg)
        self.n_bins = 0

    def close(self):
        if self.h is not None:
            lisa_like_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_data(self, f0, df, n_bins, d, psd):
        """d complex [3, n_bins] (or None), psd [3, n_bins]."""
        dd = None
        if d is not None:
            d = np.asarray(d)
            dd = _f64(np.stack([d.real, d.imag], axis=-1)) if np.iscomplexobj(d) else _f64(d)
        lisa_like_set_data(self.h, f0, df, n_bins, dd, psd)
        self.n_bins = int(n_bins)

    def loglike(self, params):
        p = _f64(np.atleast_2d(params))
        B = p.shape[0]
        lnL, dh, hh = np.empty(B), np.empty(B), np.empty(B)
        lisa_like_loglike(self.h, p, B, lnL, dh, hh)
        return lnL, dh, hh

    def data_inner(self):
        return lisa_like_data_inner(self.h)

    def template(self, params):
        out = np.empty((3, self.n_bins, 2))
        lisa_like_template(self.h, _f64(params), out)
        return out[..., 0] + 1j * out[..., 1]

    def stage_knots(self, params):
        p = _f64(np.atleast_2d(params))
        B = p.shape[0]
        band = np.empty((B, self.L, 3), dtype=np.int64)
        fedge = np.empty((B, self.L, 2))
        fk = np.empty((B, self.L, self.K))
        vals = np.empty((B, self.L, 8, self.K))
        lisa_like_stage_knots(self.h, p, B, band, fedge, fk, vals)
        return band, fedge, fk, vals

    def stage_coeffs(self, params):
        p = _f64(np.atleast_2d(params))
        B = p.shape[0]
        coef = np.empty((B, self.L, self.K - 1, 8, 4))
        lisa_like_stage_coeffs(self.h, p, B, coef)
        return coef

    def mode_inner(self, params):
        """Per-mode <d|h_i> and <h_i|h_i>, arrays [B, n_modes]."""
        p = _f64(np.atleast_2d(params))
        B = p.shape[0]
        dh = np.empty((B, self.L))
        hh = np.empty((B, self.L))
        lisa_like_mode_inner(self.h, p, B, dh, hh)
        return dh, hh

    def last_launches(self):
        return lisa_like_last_launches(self.h)

    def mode_cross(self, params):
        """Re<h_a|h_b> for every pair of modes, array [B, n_modes, n_modes]."""
        p = _f64(np.atleast_2d(params))
        B = p.shape[0]
        out = np.empty((B, self.L, self.L))
        _check(load().lisa_like_mode_cross(self.h, _ptr(p), B, _ptr(out)), self.h)
        return out

    def set_fiducial(self, params, n_rb=256):
        """Relative-binning summary data about the fiducial `params` [11]."""
        p = _f64(params)
        _check(load().lisa_like_set_fiducial(self.h, _ptr(p), int(n_rb)), self.h)

    def rb_edges(self):
        n = C.c_int()
        _check(load().lisa_like_rb_edges(self.h, None, C.byref(n)), self.h)
        e = np.empty(n.value, dtype=np.int64)
        _check(load().lisa_like_rb_edges(self.h, _ptr(e), C.byref(n)), self.h)
        return e

    def loglike_rb(self, params):
        """ln L, <d|h>, <h|h> by relative binning (after set_fiducial)."""
        p = _f64(np.atleast_2d(params))
        B = p.shape[0]
        lnL, dh, hh = np.empty(B), np.empty(B), np.empty(B)
        _check(load().lisa_like_loglike_rb(self.h, _ptr(p), B, _ptr(lnL), _ptr(dh), _ptr(hh)),
               self.h)
        return lnL, dh, hh


def dl_from_z(z):
    return np.array([lisa_dl_from_z(v) for v in np.atleast_1d(z)])


def psd_aet(f0, df, n_bins):
    out = np.empty((3, n_bins))
    lisa_psd_aet(f0, df, n_bins, out)
    return out


# ------------------------------------------------------------------- sampler (lisa_sampler.h)

def _scheck(st, s=None):
    if st != LISA_OK:
        raise LisaError(st, lisa_sampler_last_error(s))


def lisa_sampler_default_config() -> lisa_sampler_config:
    cfg = lisa_sampler_config()
    load().lisa_sampler_default_config(C.byref(cfg))
    return cfg


def lisa_sampler_create(like_h, cfg: lisa_sampler_config):
    s = C.c_void_p()
    _scheck(load().lisa_sampler_create(like_h, C.byref(cfg), C.byref(s)))
    return s


def lisa_sampler_set_ladder(s, betas):
    b = _f64(betas)
    _scheck(load().lisa_sampler_set_ladder(s, _ptr(b)), s)


def lisa_sampler_set_state(s, x, step=0):
    xx = _f64(x)
    _scheck(load().lisa_sampler_set_state(s, _ptr(xx), int(step)), s)


def lisa_sampler_run(s, n_steps, d_chain=None, d_lnl=None):
    _scheck(load().lisa_sampler_run(s, int(n_steps), _ptr(d_chain), _ptr(d_lnl)), s)


def lisa_sampler_get_state(s, x=None, lnl=None, betas=None):
    step = C.c_uint32()
    _scheck(load().lisa_sampler_get_state(s, _ptr(x), _ptr(lnl), _ptr(betas), C.byref(step)), s)
    return step.value


def lisa_sampler_get_counts(s, acc=None, swaps=None):
    _scheck(load().lisa_sampler_get_counts(s, _ptr(acc), _ptr(swaps)), s)


def lisa_sampler_step_launches(s) -> int:
    return load().lisa_sampler_step_launches(s)


def lisa_sampler_destroy(s):
    load().lisa_sampler_destroy(s)


def lisa_sampler_last_error(s=None) -> str:
    msg = load().lisa_sampler_last_error(s)
    return msg.decode() if msg else ""


def lisa_sampler_to_physical(d_x, n, lisa_frame, t0, d_th, stream=None):
    st = None if stream is None else C.c_void_p(int(stream))
    _scheck(load().lisa_sampler_to_physical(_ptr(d_x), int(n), int(bool(lisa_frame)), float(t0),
                                            _ptr(d_th), st))


def lisa_sampler_from_physical(th, n, lisa_frame, t0, x_out):
    t = _f64(th)
    _scheck(load().lisa_sampler_from_physical(_ptr(t), int(n), int(bool(lisa_frame)), float(t0),
                                              _ptr(x_out)))


def from_physical(th, lisa_frame=True, t0=3.15576e7):
    """Sampling coordinates of Table I (host) from physical parameters [n, 11] or [11]."""
    t = _f64(np.atleast_2d(th))
    out = np.empty_like(t)
    lisa_sampler_from_physical(t, t.shape[0], lisa_frame, t0, out)
    return out if np.ndim(th) == 2 else out[0]


def lisa_sampler_sky_mode_init(x_center, scale, lower, upper, T, W, seed, x_out):
    xc, sc, lo, hi = _f64(x_center), _f64(scale), _f64(lower), _f64(upper)
    _scheck(load().lisa_sampler_sky_mode_init(_ptr(xc), _ptr(sc), _ptr(lo), _ptr(hi), int(T),
                                              int(W), int(seed), _ptr(x_out)))


def lisa_autocorr_time(d_chain, n, W, stride=1, offset=0, rho=None, stream=None):
    tau = C.c_double()
    st = None if stream is None else C.c_void_p(int(stream))
    _scheck(load().lisa_autocorr_time(_ptr(d_chain), int(n), int(W), int(stride), int(offset),
                                      C.byref(tau), _ptr(rho), st))
    return tau.value


def sampler_config(**kw) -> lisa_sampler_config:
    """lisa_sampler_default_config() with fields overridden by keyword."""
    cfg = lisa_sampler_default_config()
    for k, v in kw.items():
        if k in ("lower", "upper", "gauss_mean", "gauss_sigma"):
            arr = getattr(cfg, k)
            for q, val in enumerate(np.asarray(v, dtype=np.float64).reshape(SAMPLER_NDIM)):
                arr[q] = float(val)
        else:
            setattr(cfg, k, v)
    return cfg


class LisaSampler:
    """Owns one sampler handle.  `like` is a LisaLike (or None for the Gaussian target).
    Chains come back as numpy arrays; the device buffers are torch tensors."""

    def __init__(self, like=None, **cfg):
        self.cfg = sampler_config(**cfg)
        self.T, self.W = self.cfg.n_temps, self.cfg.n_walkers
        self.like = like
        self.h = lisa_sampler_create(None if like is None else like.h, self.cfg)

    def close(self):
        if self.h is not None:
            lisa_sampler_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_ladder(self, betas):
        lisa_sampler_set_ladder(self.h, betas)

    def set_state(self, x, step=0):
        x = _f64(x).reshape(self.T, self.W, SAMPLER_NDIM)
        lisa_sampler_set_state(self.h, x, step)

    def run(self, n_steps, record=True):
        """Run n_steps; returns (chain [n, W, 11], lnl [n, W]) of the coldest temperature
        (None, None without record)."""
        import torch

        ch = lnl = None
        if record:
            dev = torch.device("cuda", torch.cuda.current_device())
            ch = torch.empty((n_steps, self.W, SAMPLER_NDIM), dtype=torch.float64, device=dev)
            lnl = torch.empty((n_steps, self.W), dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
        lisa_sampler_run(self.h, n_steps, ch, lnl)
        if not record:
            return None, None
        return ch.cpu().numpy(), lnl.cpu().numpy()

    def run_device(self, n_steps, d_chain=None, d_lnl=None):
        lisa_sampler_run(self.h, n_steps, d_chain, d_lnl)

    def state(self):
        x = np.empty((self.T, self.W, SAMPLER_NDIM))
        lnl = np.empty((self.T, self.W))
        betas = np.empty(self.T)
        step = lisa_sampler_get_state(self.h, x, lnl, betas)
        return x, lnl, betas, step

    def counts(self):
        acc = np.empty((self.T, 2), dtype=np.int64)
        sw = np.empty((self.T, 2), dtype=np.int64)
        lisa_sampler_get_counts(self.h, acc, sw)
        return acc, sw

    def step_launches(self):
        return lisa_sampler_step_launches(self.h)

    def enable_flow(self, **kw):
        """Flow proposals for the coldest temperature (lisa_flow_schedule fields as
        keywords); returns the sampler's Flow (borrowed)."""
        fs = lisa_flow_default_schedule()
        for k, v in kw.items():
            setattr(fs, k, v)
        _scheck(load().lisa_sampler_enable_flow(self.h, C.byref(fs)), self.h)
        self.flow = Flow(handle=load().lisa_sampler_get_flow(self.h))
        return self.flow

    def set_flow_likelihood(self, like2):
        """Flow proposals evaluated by another LisaLike (e.g. FP64); None restores."""
        _scheck(load().lisa_sampler_set_flow_likelihood(self.h, None if like2 is None else like2.h),
                self.h)
        self.flow_like = like2

    def set_flow_screen(self, margin):
        """Screen the flow moves with the sampler's own likelihood (margin in ln L; 0: off);
        see lisa_sampler_set_flow_screen."""
        _scheck(load().lisa_sampler_set_flow_screen(self.h, float(margin)), self.h)

    def flow_screen_count(self):
        """Flow proposals sent to the second likelihood since set_state."""
        n = C.c_int64()
        _scheck(load().lisa_sampler_flow_screen_count(self.h, C.byref(n)), self.h)
        return n.value

    def flow_stats(self):
        acc = np.zeros(2, dtype=np.int64)
        n = C.c_int()
        loss = C.c_double()
        _scheck(load().lisa_sampler_flow_stats(self.h, _ptr(acc), C.byref(n), C.byref(loss)), self.h)
        return acc, n.value, loss.value

    def checkpoint(self, path):
        """Save what a resumed run needs (walkers, ladder, next step counter, seed) to an
        .npz file; ln L is re-evaluated on restore."""
        x, _, betas, step = self.state()
        np.savez(path, x=x, betas=betas, step=np.uint32(step), seed=np.uint64(self.cfg.seed))

    def restore(self, path):
        """Continue from a checkpoint: the next steps draw the same random numbers as the
        uninterrupted run (counter-based generator keyed by the seed and the step)."""
        z = np.load(path)
        if int(z["seed"]) != int(self.cfg.seed):
            raise ValueError("checkpoint was written by a sampler with another seed")
        self.set_ladder(z["betas"])
        self.set_state(z["x"], int(z["step"]))


def sky_mode_init(x_center, scale, lower, upper, T, W, seed):
    out = np.empty((T, W, SAMPLER_NDIM))
    lisa_sampler_sky_mode_init(x_center, scale, lower, upper, T, W, seed, out)
    return out


def autocorr_time(chain, stride=1, offset=0, return_rho=False):
    """tau of Sec. III.C on the device; chain is a torch tensor or numpy array of shape
    [n, W] (stride 1) or [n, W, stride]."""
    import torch

    t = chain if hasattr(chain, "data_ptr") else torch.as_tensor(np.ascontiguousarray(chain))
    t = t.to(device="cuda", dtype=torch.float64).contiguous()
    n, W = t.shape[0], t.shape[1]
    rho = np.empty(n) if return_rho else None
    torch.cuda.synchronize()
    tau = lisa_autocorr_time(t, n, W, stride, offset, rho)
    return (tau, rho) if return_rho else tau


# ------------------------------------------------------------------- flow (lisa_flow.h)

def lisa_flow_default_schedule() -> lisa_flow_schedule:
    fs = lisa_flow_schedule()
    load().lisa_flow_default_schedule(C.byref(fs))
    return fs


def _fcheck(st, f=None):
    if st != LISA_OK:
        msg = load().lisa_flow_last_error(f)
        raise LisaError(st, msg.decode() if msg else "")


def pack_flow_weights(w) -> np.ndarray:
    """Dict of arrays (W1 [8,128,11], b1 [8,128], W2 [8,128,128], b2 [8,128],
    W3 [8,22,128], b3 [8,22]) -> the packed [8][20886] float32 layout of lisa_flow.h."""
    parts = [np.asarray(w[k], dtype=np.float32).reshape(FLOW_COUPLINGS, -1)
             for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    out = np.ascontiguousarray(np.concatenate(parts, axis=1))
    assert out.shape == (FLOW_COUPLINGS, FLOW_PARAMS_PER_COUPLING)
    return out


def unpack_flow_weights(p) -> dict:
    p = np.asarray(p, dtype=np.float32).reshape(FLOW_COUPLINGS, FLOW_PARAMS_PER_COUPLING)
    H, D = FLOW_HIDDEN, SAMPLER_NDIM
    shapes = (("W1", (H, D)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (2 * D, H)),
              ("b3", (2 * D,)))
    out, o = {}, 0
    for k, shp in shapes:
        n = int(np.prod(shp))
        out[k] = p[:, o:o + n].reshape((FLOW_COUPLINGS,) + shp).copy()
        o += n
    return out


class Flow:
    """One flow handle (owned, or borrowed from a sampler).  Device arrays are torch
    tensors of float64 rows of 11 values."""

    def __init__(self, seed=1, handle=None):
        self.own = handle is None
        if handle is None:
            h = C.c_void_p()
            _fcheck(load().lisa_flow_create(int(seed), C.byref(h)))
            handle = h.value
        self.h = C.c_void_p(handle)

    def close(self):
        if self.own and self.h is not None:
            load().lisa_flow_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, w):
        p = pack_flow_weights(w) if isinstance(w, dict) else np.ascontiguousarray(w, np.float32)
        _fcheck(load().lisa_flow_set_weights(self.h, _ptr(p)), self.h)

    def weights(self):
        p = np.empty((FLOW_COUPLINGS, FLOW_PARAMS_PER_COUPLING), np.float32)
        _fcheck(load().lisa_flow_get_weights(self.h, _ptr(p)), self.h)
        return unpack_flow_weights(p)

    def set_whitening(self, mu, L):
        """mu [11]; L [11, 11] lower triangular, or a vector of scales (diagonal L)."""
        m = _f64(mu)
        Lm = np.asarray(L, dtype=np.float64)
        Lm = _f64(np.diag(Lm) if Lm.ndim == 1 else Lm)
        _fcheck(load().lisa_flow_set_whitening(self.h, _ptr(m), _ptr(Lm)), self.h)

    set_standardisation = set_whitening

    def whitening(self):
        m, Lm = np.empty(SAMPLER_NDIM), np.empty((SAMPLER_NDIM, SAMPLER_NDIM))
        _fcheck(load().lisa_flow_get_whitening(self.h, _ptr(m), _ptr(Lm)), self.h)
        return m, Lm

    def _dev(self, a):
        import torch

        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()

    def normalize(self, x):
        import torch

        dx = self._dev(x)
        n = dx.shape[0]
        z = torch.empty_like(dx)
        lq = torch.empty(n, dtype=torch.float64, device=dx.device)
        torch.cuda.synchronize()
        _fcheck(load().lisa_flow_normalize(self.h, _ptr(dx), n, _ptr(z), _ptr(lq), None), self.h)
        torch.cuda.synchronize()
        return z.cpu().numpy(), lq.cpu().numpy()

    def generate(self, z):
        import torch

        dz = self._dev(z)
        n = dz.shape[0]
        x = torch.empty_like(dz)
        lq = torch.empty(n, dtype=torch.float64, device=dz.device)
        torch.cuda.synchronize()
        _fcheck(load().lisa_flow_generate(self.h, _ptr(dz), n, _ptr(x), _ptr(lq), None), self.h)
        torch.cuda.synchronize()
        return x.cpu().numpy(), lq.cpu().numpy()

    def gradients(self, x):
        import torch

        dx = self._dev(x)
        g = np.empty((FLOW_COUPLINGS, FLOW_PARAMS_PER_COUPLING), np.float32)
        loss = C.c_double()
        torch.cuda.synchronize()
        _fcheck(load().lisa_flow_gradients(self.h, _ptr(dx), dx.shape[0], _ptr(g),
                                           C.byref(loss), None), self.h)
        return loss.value, unpack_flow_weights(g)

    def train(self, data, iters, batch=1024, lr=1e-3, seed=1, round_=0):
        import torch

        dd = data if hasattr(data, "data_ptr") else self._dev(data)
        loss = np.empty(iters)
        torch.cuda.synchronize()
        _fcheck(load().lisa_flow_train(self.h, _ptr(dd), dd.shape[0], int(iters), int(batch),
                                       float(lr), int(seed), int(round_), _ptr(loss), None),
                self.h)
        return loss


def probe_pipes(device=0):
    """Measured FP64 FMA/s, FP32 FMA/s, MUFU sin/s of the device and its SM clock [Hz]."""
    out = (C.c_double * 4)()
    _check(load().lisa_probe_pipes(int(device), out))
    return {"fp64_fma_per_s": out[0], "fp32_fma_per_s": out[1], "mufu_per_s": out[2],
            "sm_clock_hz": out[3]}
