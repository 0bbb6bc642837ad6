"""C-ABI checks that need no GPU: the library loads, exports every function the
header declares, and reports errors without touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_01827_gb300 import build, lisalike

    build.build()
    return lisalike.load()


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(lisa_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol():
    from paper_2005_01827_gb300 import lisalike

    assert set(lisalike.SYMBOLS) == declared_functions()


def test_config_struct_layout_matches_header(lib):
    from paper_2005_01827_gb300 import lisalike

    cfg = lisalike.lisa_like_config()
    lib.lisa_like_default_config(C.byref(cfg))
    assert cfg.n_modes == 6 and cfg.n_knots == 1024 and cfg.max_batch == 1024
    assert [tuple(cfg.modes[i]) for i in range(6)] == [(2, 2), (3, 3), (4, 4), (2, 1), (3, 2), (4, 3)]
    assert cfg.t0_s == 3.15576e7 and cfg.timeout_s == 60.0 and cfg.precision == 0


def test_create_rejects_bad_configs_before_any_device_call(lib):
    from paper_2005_01827_gb300 import lisalike

    h = C.c_void_p()
    bad = []
    for mutate in (lambda c: setattr(c, "n_modes", 0), lambda c: setattr(c, "n_knots", 3),
                   lambda c: setattr(c, "precision", 7), lambda c: setattr(c, "max_batch", 0)):
        cfg = lisalike.lisa_like_default_config()
        mutate(cfg)
        bad.append(cfg)
    cfg = lisalike.lisa_like_default_config()
    cfg.modes[1][0], cfg.modes[1][1] = 2, 2          # duplicate mode
    bad.append(cfg)
    cfg = lisalike.lisa_like_default_config()
    cfg.modes[0][0], cfg.modes[0][1] = 5, 5          # not a PhenomHM mode
    bad.append(cfg)
    for cfg in bad:
        assert lib.lisa_like_create(C.byref(cfg), C.byref(h)) == lisalike.LISA_ERR_ARG
        assert lisalike.lisa_like_last_error(None) != ""
    assert lib.lisa_like_create(None, C.byref(h)) == lisalike.LISA_ERR_ARG


def test_null_handle_is_rejected(lib):
    from paper_2005_01827_gb300 import lisalike

    assert lib.lisa_like_loglike(None, None, 1, None, None, None) == lisalike.LISA_ERR_ARG
    assert lib.lisa_like_set_data(None, 1.0, 1.0, 1, None, None) == lisalike.LISA_ERR_ARG
    lib.lisa_like_destroy(None)


def test_host_helpers(lib, orc):
    from paper_2005_01827_gb300 import lisalike

    for z in (0.01, 1.0, 4.0, 7.0, 100.0):
        assert abs(lisalike.lisa_dl_from_z(z) / orc.dl_gpc(z) - 1) < 1e-9
    assert np.isnan(lisalike.lisa_dl_from_z(-1.0))
    f0, df, n = 1e-5, 1e-6, 5000
    out = lisalike.psd_aet(f0, df, n)
    ref = orc.psd_aet(f0 + df * np.arange(n))
    assert np.allclose(out, ref, rtol=1e-12, atol=0)


def test_sampler_host_functions_match_the_oracle(lib, orc):
    """Host-only entry points of include/lisa_sampler.h, callable without a GPU."""
    import math

    import workloads as W
    from paper_2005_01827_gb300 import lisalike as LL

    rng = np.random.default_rng(3)
    th = W.draw_walkers(64, 4, (3.0, 9.0))
    th[:, 4] = rng.uniform(0.1, 100.0, 64)
    th[:, 10] = rng.uniform(600.0, 1e7, 64)
    for frame in (False, True):
        x = LL.from_physical(th, frame, W.T0_YEAR)
        for v, t in zip(x, th):
            ref = orc.from_physical(t)
            if frame:
                tL, lamL, betL, psiL = orc.ssb_to_lisa(t[10] + W.T0_YEAR, t[7], t[8], t[9])
                ref[7], ref[8], ref[9], ref[10] = lamL, math.sin(betL), psiL, math.log(tL - W.T0_YEAR)
            d = np.abs(v - ref)
            d[7] = abs((v[7] - ref[7] + math.pi) % (2 * math.pi) - math.pi)
            d[9] = abs((v[9] - ref[9] + math.pi / 2) % math.pi - math.pi / 2)
            assert np.max(d) <= 1e-11, (frame, d)
    with pytest.raises(LL.LisaError):
        LL.from_physical(np.where(np.arange(11) == 0, -1.0, th[0]), False, 0.0)
    # sky-mode initialisation: 8 modes, W/8 walkers each, inside the prior box
    c = LL.lisa_sampler_default_config()
    lo, hi = np.array(list(c.lower)), np.array(list(c.upper))
    xc = LL.from_physical(th[0], True, W.T0_YEAR)
    x0 = LL.sky_mode_init(xc, np.full(11, 1e-6), lo, hi, 3, 32, 9)
    assert np.all(x0 >= lo) and np.all(x0 <= hi)
    for w in range(32):
        lam = (xc[7] + (w % 4) * math.pi / 2 - lo[7]) % (hi[7] - lo[7]) + lo[7]
        assert abs((x0[1, w, 7] - lam + math.pi) % (2 * math.pi) - math.pi) <= 1e-4
        assert abs(x0[1, w, 8] - (xc[8] if w % 8 < 4 else -xc[8])) <= 1e-4
    assert not np.array_equal(x0[0], x0[1])           # independent jitter per temperature
    with pytest.raises(LL.LisaError):
        LL.sky_mode_init(xc, np.full(11, 1e-6), lo, hi, 1, 12, 9)   # W not a multiple of 8
