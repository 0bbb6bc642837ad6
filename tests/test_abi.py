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
