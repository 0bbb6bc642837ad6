"""Uneven batches under CUDA-graph replay with autotuned tile shapes (the 8192-walker
workload: masses log-uniform over 1e3..1e9 Msun, so mode bands differ by orders of
magnitude), against the FP64 oracle on sampled walkers."""
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


def test_graph_replay_equals_direct_calls(pkg, orc):
    import torch

    LL = pkg.lisalike
    g = W.Grid.spanning(1e-4, 2e-2, 1.0 / (30 * W.DAY_S))
    th = W.draw_walkers(40, 12, (3.0, 9.0))
    th[:, 4] = [orc.dl_gpc(z) for z in th[:, 4]]
    S = orc.psd_aet(g.freqs())
    d = orc.template(th[3], W.T0_C1, W.MODES6, 64, g.f0, g.df, g.n_bins)
    for prec in (pkg.LISA_PREC_FP64, pkg.LISA_PREC_SPLIT):
        like = pkg.LisaLike(modes=W.MODES6, n_knots=64, t0=W.T0_C1, max_batch=40, precision=prec)
        like.set_data(g.f0, g.df, g.n_bins, d, S)
        ref, _, _ = like.loglike(th)
        LL.lisa_like_set_graphs(like.h, True)
        a, _, _ = like.loglike(th)           # capture + replay
        b, _, _ = like.loglike(th)           # replay
        assert np.array_equal(a, ref) and np.array_equal(b, ref)
        dp = torch.tensor(th, dtype=torch.float64, device="cuda")
        out = torch.empty(40, dtype=torch.float64, device="cuda")
        st = torch.cuda.Stream()
        for _ in range(2):                   # new pointers: re-capture, then replay
            LL.lisa_like_loglike_device(like.h, dp, 40, out, None, None, st.cuda_stream)
            st.synchronize()
            assert np.array_equal(out.cpu().numpy(), ref)
        assert like.last_launches() == 8
        like.close()


def test_autotune_picks_a_supported_shape_and_keeps_results(pkg, orc):
    LL = pkg.lisalike
    g = W.Grid.spanning(1e-4, 2e-2, 1.0 / (30 * W.DAY_S))
    th = W.draw_walkers(24, 13, (3.0, 9.0))
    th[:, 4] = [orc.dl_gpc(z) for z in th[:, 4]]
    S = orc.psd_aet(g.freqs())
    d = orc.template(th[0], W.T0_C1, W.MODES6, 64, g.f0, g.df, g.n_bins)
    for prec in (pkg.LISA_PREC_FP64, pkg.LISA_PREC_SPLIT):
        like = pkg.LisaLike(modes=W.MODES6, n_knots=64, t0=W.T0_C1, max_batch=24, precision=prec)
        like.set_data(g.f0, g.df, g.n_bins, d, S)
        shape = LL.lisa_like_autotune(like.h, th, 24)
        assert shape[:2] in ((8, 8), (4, 8), (16, 8), (8, 1)) and shape[2] > 0
        assert LL.lisa_like_autotune(like.h, th, 24) == shape     # cached
        lnL, _, hh = like.loglike(th)
        ref, _, rhh, dd = orc.loglike(th, W.T0_C1, W.MODES6, 64, g.f0, g.df, d, S)
        scale = np.maximum(np.maximum(rhh, dd), 1.0)
        fin = np.isfinite(ref)
        assert np.all(np.abs(lnL - ref)[fin] <= 1e-6 * scale[fin])
        # another tile shape changes only the summation order: FP64 rounding, or the
        # FP32 partial sums of split precision
        tol = 1e-9 if prec == pkg.LISA_PREC_FP64 else 1e-6
        for shp in ((8, 1), (4, 8)):
            LL.lisa_like_set_tune(like.h, *shp)
            other, _, _ = like.loglike(th)
            assert np.all(np.abs(other - lnL)[fin] <= tol * scale[fin])
        with pytest.raises(LL.LisaError):
            LL.lisa_like_set_tune(like.h, 3, 3)
        like.close()


@pytest.fixture(scope="module")
def c3_case(orc):
    """The 8192-walker workload's data and walkers, and the oracle on 128+ of them
    (the 8 lightest and 8 heaviest, bands at the grid edges, random picks)."""
    from fullsize import sample_walkers

    g = W.GRID_C2
    S = orc.psd_aet(g.freqs())
    inj = W.theta_table2(1)
    d = orc.template(inj, W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, g.n_bins)
    d = d + orc.noise(S, g.df, W.white_noise(g.n_bins, 2))
    th = W.draw_walkers_c3(8192, 3)
    th[:, 4] = [orc.dl_gpc(z) for z in th[:, 4]]
    idx, n_edge = sample_walkers(orc, th, W.T0_YEAR, W.MODES6, g, seed=1)
    ref, rdh, rhh, dd = orc.loglike(th[idx], W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, d, S)
    return g, S, d, th, idx, n_edge, ref, rhh, dd


@pytest.mark.parametrize("split", [False, True])
def test_8192_walkers_masses_1e3_to_1e9(pkg, c3_case, split):
    """The 8192-walker workload at full size: graph-captured, autotuned, FP64 and split
    precision, against the oracle on the sampled walkers."""
    LL = pkg.lisalike
    g, S, d, th, idx, n_edge, ref, rhh, dd = c3_case
    assert idx.size >= 128
    prec = pkg.LISA_PREC_SPLIT if split else pkg.LISA_PREC_FP64
    like = pkg.LisaLike(modes=W.MODES6, n_knots=1024, max_batch=8192, precision=prec)
    like.set_data(g.f0, g.df, g.n_bins, d, S)
    LL.lisa_like_autotune(like.h, th[:256], 256)
    LL.lisa_like_set_graphs(like.h, True)
    lnL, dh, hh = like.loglike(th)
    again, _, _ = like.loglike(th)          # replay of the captured graph
    like.close()
    assert np.all(np.isfinite(lnL)) and np.array_equal(again, lnL)
    m = th[:, 0]
    scale = np.maximum(np.maximum(rhh, dd), 1.0)
    err = np.abs(lnL[idx] - ref) / scale
    sig = rhh > 1e-6
    rel_hh = np.abs(hh[idx] - rhh)[sig] / rhh[sig]
    print("8192-walker %s, %d walkers (%d at grid edges, masses %.3g..%.3g): max |d lnL| / "
          "SNR^2 = %.3e, max |d lnL| = %.3e, max rel d<h|h> = %.3e"
          % ("split" if split else "fp64", idx.size, n_edge, m[idx].min(), m[idx].max(),
             err.max(), np.abs(lnL[idx] - ref).max(), rel_hh.max()))
    assert np.all(err <= 1e-6)
    assert np.all(rel_hh <= 1e-6)
