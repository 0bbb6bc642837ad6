"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by
element on the intermediate stages and on ln L, <d|h>, <h|h>.

Tolerances: stage values agree to ~1e-9 relative (different transcendental
implementations, FMA contraction); ln L must meet |d lnL| <= 1e-6 SNR^2 in FP64 mode
(the stated requirement), where SNR^2 = max(<d|d>_signal, <h|h>) of the walker.
"""
import math
import os

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


def c1_setup(orc):
    g = W.GRID_C1
    th = np.array(W.THETA_C1_Z, dtype=float)
    th[4] = orc.dl_gpc(th[4])
    S = orc.psd_aet(g.freqs())
    d = orc.template(th, W.T0_C1, [(2, 2)], 256, g.f0, g.df, g.n_bins)
    return g, th, S, d


def walkers(orc, B, seed, logm=(5.0, 7.0)):
    th = W.draw_walkers(B, seed, logm)
    th[:, 4] = [orc.dl_gpc(z) for z in th[:, 4]]
    return th


# ----------------------------------------------------------------------------- stages

def test_c1_knot_stage_matches_oracle(pkg, orc):
    g, th, S, d = c1_setup(orc)
    like = pkg.LisaLike(modes=[(2, 2)], n_knots=256, t0=W.T0_C1, max_batch=2)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    band, fedge, fk, vals = like.stage_knots(th)
    flo, fhi, jlo, jhi = orc.band(th, W.T0_C1, 2, 2, g.f0, g.df, g.n_bins)
    assert band[0, 0].tolist() == [1, jlo, jhi]
    assert abs(fedge[0, 0, 0] - flo) <= 1e-13 * flo and fedge[0, 0, 1] == fhi
    rfk, rvals = orc.knots(th, W.T0_C1, 2, 2, g.f0, g.df, g.n_bins, 256)
    assert np.allclose(fk[0, 0], rfk, rtol=1e-13, atol=0)
    for q in range(8):
        scale = np.max(np.abs(rvals[q]))
        assert np.max(np.abs(vals[0, 0, q] - rvals[q])) <= 1e-9 * scale, q
    like.close()


def test_multimode_stages_match_oracle(pkg, orc):
    g = W.Grid.spanning(1e-4, 2e-2, 1.0 / (30 * W.DAY_S))
    th = walkers(orc, 6, 21)
    S = orc.psd_aet(g.freqs())
    K = 64
    like = pkg.LisaLike(modes=W.MODES6, n_knots=K, t0=W.T0_C1, max_batch=8)
    like.set_data(g.f0, g.df, g.n_bins, None, S)
    band, fedge, fk, vals = like.stage_knots(th)
    coef = like.stage_coeffs(th)
    for b in range(th.shape[0]):
        for mi, (l, m) in enumerate(W.MODES6):
            ref = orc.band(th[b], W.T0_C1, l, m, g.f0, g.df, g.n_bins)
            if ref is None:
                assert band[b, mi, 0] == 0
                continue
            assert band[b, mi].tolist() == [1, ref[2], ref[3]]
            rfk, rvals = orc.knots(th[b], W.T0_C1, l, m, g.f0, g.df, g.n_bins, K)
            assert np.allclose(fk[b, mi], rfk, rtol=1e-12, atol=0)
            for q in range(8):
                scale = np.max(np.abs(rvals[q])) + 1e-300
                assert np.max(np.abs(vals[b, mi, q] - rvals[q])) <= 1e-9 * scale
                # the interpolants agree inside every segment (raw cubic coefficients
                # amplify knot-value rounding by 1/h^3, the interpolant does not)
                rc = orc.spline(rfk, rvals[q])
                hseg = np.diff(rfk)
                for frac in (0.0, 1.0 / 3.0, 2.0 / 3.0, 1.0):
                    x = (frac * hseg)[:, None] ** np.arange(4)[None, :]
                    got = np.sum(coef[b, mi, :, q, :] * x, axis=1)
                    want = np.sum(rc * x, axis=1)
                    assert np.max(np.abs(got - want)) <= 1e-8 * scale, (b, mi, q, frac)
    like.close()


def test_c1_template_matches_oracle(pkg, orc):
    g, th, S, d = c1_setup(orc)
    like = pkg.LisaLike(modes=[(2, 2)], n_knots=256, t0=W.T0_C1, max_batch=1)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    h = like.template(th)
    assert np.max(np.abs(h - d)) <= 1e-8 * np.max(np.abs(d))
    like.close()


# ----------------------------------------------------------------------------- ln L

def test_c1_noise_free_injection(pkg, orc):
    g, th, S, d = c1_setup(orc)
    like = pkg.LisaLike(modes=[(2, 2)], n_knots=256, t0=W.T0_C1, max_batch=4)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    snr2 = orc.inner(d, d, S, g.df)
    assert abs(like.data_inner() - snr2) <= 1e-12 * snr2
    lnL, dh, hh = like.loglike(th)
    assert abs(lnL[0]) <= 1e-6 * snr2          # ln L(theta0) = 0
    assert abs(hh[0] - snr2) <= 1e-6 * snr2    # <h|h> = SNR^2
    assert abs(lnL[0]) <= 1e-9 * snr2          # and in fact to ~rounding
    like.close()


def _compare(like, orc, th, t0, modes, K, g, d, S, tol_rel=1e-6):
    lnL, dh, hh = like.loglike(th)
    ref, rdh, rhh, dd = orc.loglike(th, t0, modes, K, g.f0, g.df, d, S)
    ok = np.isfinite(ref)
    assert np.array_equal(np.isneginf(lnL), np.isneginf(ref))
    scale = np.maximum(np.maximum(dd, rhh), 1.0)
    err = np.abs(lnL - ref)[ok] / scale[ok]
    assert np.all(err <= tol_rel), (err.max(), np.argmax(err))
    assert np.all(np.abs(hh - rhh)[ok] <= tol_rel * scale[ok])
    assert np.all(np.abs(dh - rdh)[ok] <= tol_rel * scale[ok])
    return err.max() if err.size else 0.0


def test_batched_six_modes_ragged(pkg, orc):
    """Several tiles per walker, ragged tails, bands that start mid-grid, noise."""
    g = W.Grid.spanning(1e-4, 2e-2, 1.0 / (30 * W.DAY_S))
    t0 = W.T0_C1
    th = walkers(orc, 24, 5)
    th[:, 10] = np.linspace(-2e5, 2e5, th.shape[0])
    S = orc.psd_aet(g.freqs())
    inj = th[0].copy()
    d = orc.template(inj, t0, W.MODES6, 128, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 9))
    like = pkg.LisaLike(modes=W.MODES6, n_knots=128, t0=t0, max_batch=32)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    err = _compare(like, orc, th, t0, W.MODES6, 128, g, d, S)
    assert err < 1e-9
    like.close()


def test_edge_cases(pkg, orc):
    g, th, S, d = c1_setup(orc)
    t0 = W.T0_C1
    like = pkg.LisaLike(modes=[(2, 2), (3, 3)], n_knots=4, t0=t0, max_batch=8)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    dd = like.data_inner()
    B = np.repeat(th[None, :], 6, axis=0)
    B[1, 1] = 1.2            # invalid q
    B[2, 0] = 1e9            # band entirely below the grid: h = 0
    B[3, 10] = 1e9           # merges long after the window: band starts at the grid edge
    B[4, 0] = 30.0           # tiny mass: band beyond the grid start
    B[5, 1] = 1.0            # equal mass: odd-m mode vanishes
    lnL, dh, hh = like.loglike(B)
    ref, _, rhh, _ = orc.loglike(B, t0, [(2, 2), (3, 3)], 4, g.f0, g.df, d, S)
    assert np.isneginf(lnL[1]) and np.isneginf(ref[1])
    assert lnL[2] == pytest.approx(-0.5 * dd, rel=1e-12) and hh[2] == 0.0
    fin = np.isfinite(ref)
    scale = np.maximum(np.maximum(rhh, dd), 1.0)
    assert np.all(np.abs(lnL[fin] - ref[fin]) <= 1e-6 * scale[fin])
    like.close()
    # grids of one, two and seven bins inside the inspiral
    f0 = 1e-3
    for n in (1, 2, 7):
        like = pkg.LisaLike(modes=[(2, 2)], n_knots=8, t0=t0, max_batch=2)
        Sn = orc.psd_aet(f0 + g.df * np.arange(n))
        like.set_data(f0, g.df, n, None, Sn)
        lnL, _, hh = like.loglike(th)
        ref, _, rhh, _ = orc.loglike(th, t0, [(2, 2)], 8, f0, g.df, np.zeros((3, n), complex), Sn)
        assert np.allclose(hh, rhh, rtol=1e-9, atol=1e-300)
        assert np.allclose(lnL, ref, rtol=1e-9, atol=1e-300)
        like.close()


@pytest.mark.parametrize("split", [False, True])
def test_phase_stays_exact_along_long_segments(pkg, orc, split):
    """With d = i h, <d|h> vanishes in exact arithmetic and is first order in any phase
    error of the dense evaluation; K = 16 knots over the 1-yr grid makes segments of
    ~1e6 bins, so a phase recurrence that drifts along a segment shows up here."""
    g = W.GRID_C2
    th = W.theta_table2(1)
    th[0] = 1e5                       # band reaching the top of the grid
    K = 16
    S = orc.psd_aet(g.freqs())
    h = orc.template(th, W.T0_YEAR, [(2, 2)], K, g.f0, g.df, g.n_bins)
    like = pkg.LisaLike(modes=[(2, 2)], n_knots=K, max_batch=1,
                        precision=pkg.LISA_PREC_SPLIT if split else pkg.LISA_PREC_FP64)
    like.set_data(g.f0, g.df, g.n_bins, 1j * h, S)
    band, _, fk, _ = like.stage_knots(th)
    widest = np.max(np.diff(fk[0, 0])) / g.df
    assert widest > 5e5
    lnL, dh, hh = like.loglike(th)
    like.close()
    # FP64 resolves a phase of ~1e7 rad to ~2e-9 rad (the oracle's own per-bin rounding);
    # a recurrence drifting along these segments would give O(1e-1)
    tol = 1e-6 if split else 1e-8
    print("long segments (%.0f bins): |<i h|h>| / <h|h> = %.2e" % (widest, abs(dh[0]) / hh[0]))
    assert abs(dh[0]) <= tol * hh[0]
    assert abs(hh[0] / orc.inner(h, h, S, g.df) - 1) <= (1e-6 if split else 1e-10)


def test_errors_and_state(pkg, orc):
    from paper_2005_01827_gb300 import lisalike as LL

    g, th, S, d = c1_setup(orc)
    like = pkg.LisaLike(modes=[(2, 2)], n_knots=16, t0=W.T0_C1, max_batch=2)
    with pytest.raises(LL.LisaError) as e:
        like.loglike(th)
    assert e.value.status == LL.LISA_ERR_STATE
    bad = S.copy()
    bad[1, 7] = -1.0
    with pytest.raises(LL.LisaError) as e:
        like.set_data(g.f0, g.df, g.n_bins, d, bad)
    assert e.value.status == LL.LISA_ERR_ARG
    with pytest.raises(LL.LisaError) as e:
        like.set_data(g.f0, -1.0, g.n_bins, d, S)
    assert e.value.status == LL.LISA_ERR_ARG
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    with pytest.raises(LL.LisaError) as e:
        like.loglike(np.repeat(th[None], 3, axis=0))   # B > max_batch
    assert e.value.status == LL.LISA_ERR_ARG
    like.close()


def test_bounded_wait_reports_timeout_and_handle_recovers(pkg, orc):
    """A host wait whose bound runs out returns LISA_ERR_TIMEOUT (no device fault)."""
    from paper_2005_01827_gb300 import lisalike as LL

    g = W.GRID_C2
    S = orc.psd_aet(g.freqs())
    th = walkers(orc, 64, 3)
    like = pkg.LisaLike(modes=W.MODES6, n_knots=1024, max_batch=64, timeout_s=1e-7)
    with pytest.raises(LL.LisaError) as e:
        like.set_data(g.f0, g.df, g.n_bins, None, S)
        like.loglike(th)
    assert e.value.status == LL.LISA_ERR_TIMEOUT
    import torch
    torch.cuda.synchronize()
    like.close()


@pytest.mark.parametrize("split", [False, True])
def test_device_wait_gives_up_and_handle_recovers(pkg, orc, split):
    """The dense kernels' bounded wait on the staging barrier: with the test switch the
    barrier is armed but no copy is issued, so every wait gives up after 64 polls with
    nothing in flight.  The host call returns LISA_ERR_TIMEOUT, the device call leaves
    NaN outputs, and the next normal call on the same handle (also under graph replay)
    is correct again."""
    import torch

    from paper_2005_01827_gb300 import lisalike as LL

    g, th, S, d = c1_setup(orc)
    prec = pkg.LISA_PREC_SPLIT if split else pkg.LISA_PREC_FP64
    like = pkg.LisaLike(modes=[(2, 2)], n_knots=256, t0=W.T0_C1, max_batch=4, precision=prec)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    P = np.stack([th, th * np.array([1.0005] + [1.0] * 10)])
    ref, _, _ = like.loglike(P)
    for graphs in (False, True):
        LL.lisa_like_set_graphs(like.h, graphs)
        LL.lisa_like_test_device_wait(like.h, 64)
        with pytest.raises(LL.LisaError) as e:
            like.loglike(P)
        assert e.value.status == LL.LISA_ERR_TIMEOUT
        dp = torch.tensor(P, dtype=torch.float64, device="cuda")
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        st = torch.cuda.Stream()
        LL.lisa_like_loglike_device(like.h, dp, 2, out, None, None, st.cuda_stream)
        st.synchronize()
        assert np.all(np.isnan(out.cpu().numpy()))
        LL.lisa_like_test_device_wait(like.h, 0)
        again, _, _ = like.loglike(P)
        assert np.array_equal(again, ref)
    with pytest.raises(LL.LisaError) as e:
        LL.lisa_like_test_device_wait(like.h, -1)
    assert e.value.status == LL.LISA_ERR_ARG
    like.close()


def test_device_api_matches_host_api_and_is_deterministic(pkg, orc):
    import torch

    g, th, S, d = c1_setup(orc)
    like = pkg.LisaLike(modes=[(2, 2)], n_knots=256, t0=W.T0_C1, max_batch=16)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    B = 16
    P = th[None, :] * (1.0 + 1e-4 * np.random.default_rng(0).standard_normal((B, 11)))
    lnL1, _, _ = like.loglike(P)
    lnL2, _, _ = like.loglike(P)
    assert np.array_equal(lnL1, lnL2)
    dp = torch.tensor(P, dtype=torch.float64, device="cuda")
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    pkg.lisalike.lisa_like_loglike_device(like.h, dp, B, out, None, None, s.cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), lnL1)
    assert like.last_launches() >= 5
    like.close()


# ----------------------------------------------------------------------------- full size

@pytest.fixture(scope="module")
def c2_data(orc):
    g = W.GRID_C2
    S = orc.psd_aet(g.freqs())
    inj = W.theta_table2(1)
    d = orc.template(inj, W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 2))
    return g, S, d, inj


def test_c2_full_size_sampled_walkers(pkg, orc, c2_data):
    """1024 walkers, 6 modes, K = 1024, 3.16e6 bins (the benchmark launch) in FP64 and in
    split precision; the oracle recomputes 128+ walkers one by one (the lightest, the
    heaviest, bands at the grid edges, random picks)."""
    from fullsize import sample_walkers

    g, S, d, inj = c2_data
    th = walkers(orc, 1024, 1)
    th[0] = inj
    idx, n_edge = sample_walkers(orc, th, W.T0_YEAR, W.MODES6, g)
    idx = np.union1d(idx, [0])
    assert idx.size >= 128
    ref, rdh, rhh, dd = orc.loglike(th[idx], W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, d, S)
    scale = np.maximum(dd, rhh)
    for prec in (pkg.LISA_PREC_FP64, pkg.LISA_PREC_SPLIT):
        like = pkg.LisaLike(modes=W.MODES6, n_knots=1024, max_batch=1024, precision=prec)
        like.set_data(g.f0, g.df, g.n_bins, d, S)
        pkg.lisalike.lisa_like_autotune(like.h, th[:256], 256)
        lnL, dh, hh = like.loglike(th)
        like.close()
        assert np.all(np.isfinite(lnL))
        err = np.abs(lnL[idx] - ref) / scale
        sig = rhh > 1e-6
        rel_hh = np.abs(hh[idx] - rhh)[sig] / rhh[sig]
        print("C2 %s, %d walkers (%d at grid edges): max |d lnL| / SNR^2 = %.3e, max |d lnL| "
              "= %.3e, max rel d<h|h> = %.3e" % ("fp64" if prec == pkg.LISA_PREC_FP64 else "split",
                                                 idx.size, n_edge, err.max(),
                                                 np.abs(lnL[idx] - ref).max(), rel_hh.max()))
        assert np.all(err <= 1e-6)
        assert rel_hh.max() <= 1e-6
        if prec == pkg.LISA_PREC_FP64:
            snr_inj = math.sqrt(hh[0])
            assert 200 < snr_inj < 2000
