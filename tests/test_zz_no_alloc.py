"""The allocation-free entry point lisa_like_loglike_noalloc, for callers that cannot
call cudaMalloc (code inside a framework that owns the device heap, or loops that cannot
take an allocation's device synchronisation).  Its results must equal those of the
handle-based entry point on the same inputs, on two calls in a row that reuse the one
static scratch array, without the free device memory changing.

This file is named to be collected last."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2005_01827_gb300 import build, lisalike

    build.build()
    return torch, lisalike


def staged_bins(torch, d, S, df):
    """[N][9] device layout of the no-alloc entry: w_A, w_E, w_T, (w d) re/im per channel."""
    w = torch.tensor(4.0 * df / S, dtype=torch.float64, device="cuda")          # [3, N]
    dr = torch.tensor(np.ascontiguousarray(d.real), dtype=torch.float64, device="cuda")
    di = torch.tensor(np.ascontiguousarray(d.imag), dtype=torch.float64, device="cuda")
    cols = [w[0], w[1], w[2]]
    for c in range(3):
        cols += [w[c] * dr[c], w[c] * di[c]]
    return torch.stack(cols, dim=1).contiguous()


def run_case(env, orc, grid, modes, K, th, t0):
    torch, LL = env
    S = orc.psd_aet(grid.freqs())
    d = orc.template(th[0], t0, modes, K, grid.f0, grid.df, grid.n_bins)
    d = d + orc.noise(S, grid.df, W.white_noise(grid.n_bins, 4))
    like = LL.LisaLike(modes=modes, n_knots=K, t0=t0, max_batch=th.shape[0])
    like.set_data(grid.f0, grid.df, grid.n_bins, d, S)
    ref, rdh, rhh = like.loglike(th)
    dd = like.data_inner()
    like.close()

    cfg = LL.lisa_like_default_config()
    cfg.n_modes = len(modes)
    for k, (l, m) in enumerate(modes):
        cfg.modes[k][0], cfg.modes[k][1] = l, m
    cfg.n_knots, cfg.t0_s = K, t0
    B = th.shape[0]
    bins = staged_bins(torch, d, S, grid.df)
    P = torch.tensor(th, dtype=torch.float64, device="cuda")
    outs = []
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0 = None
    for call in range(3):
        lnL = torch.full((B,), np.nan, dtype=torch.float64, device="cuda")
        dh = torch.full((B,), np.nan, dtype=torch.float64, device="cuda")
        hh = torch.full((B,), np.nan, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        if call == 1:
            free0 = torch.cuda.mem_get_info()[0]
        LL.lisa_like_loglike_noalloc(cfg, grid.f0, grid.df, grid.n_bins, bins, dd, P, B, lnL, dh,
                                     hh, stream.cuda_stream)
        stream.synchronize()
        if call >= 1:
            outs.append((lnL.cpu().numpy(), dh.cpu().numpy(), hh.cpu().numpy()))
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, "device memory changed across no-alloc calls"
    scale = np.maximum(np.maximum(rhh, dd), 1.0)
    for lnL, dh, hh in outs:      # two calls in a row, each against the handle entry point
        assert np.all(np.abs(lnL - ref) <= 1e-6 * scale)
        assert np.all(np.abs(dh - rdh) <= 1e-6 * scale)
        assert np.all(np.abs(hh - rhh) <= 1e-6 * scale)
    assert np.array_equal(outs[0][0], outs[1][0])


def test_noalloc_matches_handle_entry_point_multimode(env, orc):
    g = W.Grid.spanning(1e-4, 2e-2, 1.0 / (30 * W.DAY_S))
    th = W.draw_walkers(2, 8)
    th[:, 4] = [orc.dl_gpc(z) for z in th[:, 4]]
    run_case(env, orc, g, W.MODES6, 512, th, W.T0_C1)


def test_noalloc_matches_handle_entry_point_full_grid(env, orc):
    th = W.theta_table2(1)[None, :]
    run_case(env, orc, W.GRID_C2, W.MODES6, 1024, th, W.T0_YEAR)


def test_noalloc_rejects_requests_beyond_its_limits(env):
    """Each rejected request is sized so that, were the limit check ever loosened, the
    call would still stay inside its buffers (a failure, not an out-of-bounds access)."""
    torch, LL = env
    cfg = LL.lisa_like_default_config()          # six modes, K = 1024
    g = W.Grid(1e-4, 1e-6, 64)
    bins = torch.zeros((g.n_bins, 9), dtype=torch.float64, device="cuda")
    P = torch.zeros((2, 11), dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(LL.LisaError) as e:      # 2 x 6 x 1024 > 8192
        LL.lisa_like_loglike_noalloc(cfg, g.f0, g.df, g.n_bins, bins, 0.0, P, 2, out)
    assert e.value.status == LL.LISA_ERR_ARG and "8192" in str(e.value)
    cfg.n_modes, cfg.n_knots = 1, 4
    B, n_bins = 2048, 8192                       # 2048 x 4 knots = 8192 (allowed)
    bins = torch.zeros((n_bins, 9), dtype=torch.float64, device="cuda")
    P = torch.zeros((B, 11), dtype=torch.float64, device="cuda")
    out = torch.zeros(B, dtype=torch.float64, device="cuda")
    with pytest.raises(LL.LisaError) as e:      # 2048 x (9 + 1) items > 16384
        LL.lisa_like_loglike_noalloc(cfg, 1e-4, 1e-6, n_bins, bins, 0.0, P, B, out)
    assert e.value.status == LL.LISA_ERR_ARG and "16384" in str(e.value)
    with pytest.raises(ValueError):             # a short output buffer never reaches C
        LL.lisa_like_loglike_noalloc(cfg, 1e-4, 1e-6, 64, bins, 0.0, P, B, out[:8])
