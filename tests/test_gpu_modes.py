"""Per-mode inner products (the Table III breakdown, each harmonic's template alone)
against the oracle's single-mode templates, and their exact relation to the full
likelihood: the template is a sum over modes, so sum_i <d|h_i> = <d|h>."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2005_01827_gb300 import build

    build.build()
    import paper_2005_01827_gb300 as p

    return p


@pytest.mark.parametrize("prec", [0, 1])
def test_mode_inner_matches_oracle_single_mode_templates(pkg, orc, prec):
    g = W.GRID_C2
    S = orc.psd_aet(g.freqs())
    inj = W.theta_table2(1)
    d = orc.template(inj, W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 2))
    th = np.vstack([inj, W.theta_table2(4), W.theta_table2(6)])
    like = pkg.LisaLike(modes=W.MODES6, n_knots=1024, max_batch=4, precision=prec)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    dhm, hhm = like.mode_inner(th)
    lnL, dh, hh = like.loglike(th)
    like.close()
    # linearity in the modes (exact up to rounding; split sums in FP32 per item)
    tol_lin = 1e-11 if prec == 0 else 1e-6
    assert np.all(np.abs(dhm.sum(axis=1) - dh) <= tol_lin * np.maximum(hh, 1.0))
    for b in range(th.shape[0]):
        for i, md in enumerate(W.MODES6):
            h = orc.template(th[b], W.T0_YEAR, [md], 1024, g.f0, g.df, g.n_bins)
            rhh = orc.inner(h, h, S, g.df)
            rdh = orc.inner(d, h, S, g.df)
            scale = max(rhh, 1.0)
            assert abs(hhm[b, i] - rhh) <= 1e-6 * scale, (b, md)
            assert abs(dhm[b, i] - rdh) <= 1e-6 * max(scale, abs(rdh)), (b, md)


def test_table3_breakdown_with_the_stand_in(pkg, orc):
    """The Table III analogue for the Table II binaries (stand-in waveform; printed for
    the design notes).  The paper's ordering for Binary 1 holds."""
    g = W.GRID_C2
    S = orc.psd_aet(g.freqs())
    like = pkg.LisaLike(modes=W.MODES6, n_knots=1024, max_batch=5)
    like.set_data(g.f0, g.df, g.n_bins, None, S)
    th = np.vstack([W.theta_table2(k) for k in (1, 4, 5, 6, 7)])
    _, hhm = like.mode_inner(th)
    _, _, hh = like.loglike(th)
    like.close()
    for k, row, tot in zip((1, 4, 5, 6, 7), np.sqrt(hhm), np.sqrt(hh)):
        print("Binary %d: all %.0f  modes %s" % (k, tot, " ".join("%.1f" % v for v in row)))
    b1 = np.sqrt(hhm[0])
    assert np.argsort(-b1).tolist() == [0, 1, 2, 3, 4, 5]
    assert 300 < math.sqrt(hh[0]) < 1200


@pytest.mark.parametrize("prec", [0, 1])
def test_mode_cross_terms_match_the_oracle_and_rebuild_lnl(pkg, orc, prec):
    """Re<h_a|h_b> of every mode pair against the oracle's single-mode templates; with
    <d|h_a> it rebuilds ln L exactly (the mode-by-mode form with cross terms); the cross
    terms are why the total SNR is not the quadrature sum of the mode SNRs (Table III)."""
    g = W.GRID_C2
    S = orc.psd_aet(g.freqs())
    inj = W.theta_table2(1)
    d = orc.template(inj, W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 2))
    th = np.vstack([inj, W.theta_table2(6)])
    like = pkg.LisaLike(modes=W.MODES6, n_knots=1024, max_batch=4, precision=prec)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    X = like.mode_cross(th)
    dhm, hhm = like.mode_inner(th)
    lnL, dh, hh = like.loglike(th)
    dd = like.data_inner()
    like.close()
    tol = 1e-9 if prec == 0 else 1e-6
    for b in range(2):
        assert np.allclose(X[b], X[b].T, rtol=0, atol=0)
        assert np.allclose(np.diag(X[b]), hhm[b], rtol=0, atol=tol * hh[b])
        assert abs(X[b].sum() - hh[b]) <= tol * hh[b]
        rebuilt = dhm[b].sum() - 0.5 * X[b].sum() - 0.5 * dd
        assert abs(rebuilt - lnL[b]) <= tol * max(hh[b], dd)
        hs = [orc.template(th[b], W.T0_YEAR, [md], 1024, g.f0, g.df, g.n_bins) for md in W.MODES6]
        for a in range(6):
            for c in range(a + 1, 6):
                ref = orc.inner(hs[a], hs[c], S, g.df)
                assert abs(X[b, a, c] - ref) <= 1e-6 * hh[b], (b, a, c, X[b, a, c], ref)
    off = X[0].sum() - np.trace(X[0])
    print("Binary 1: SNR %.1f, quadrature sum of mode SNRs %.1f, cross terms %.3e of <h|h>"
          % (np.sqrt(hh[0]), np.sqrt(np.trace(X[0])), off / hh[0]))
    assert abs(off) > 1e-6 * hh[0]
