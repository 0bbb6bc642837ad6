"""Host-side logic of bench.py that decides whether a measurement stands: the clock and
throttle-reason summary taken from nvidia-smi samples during the timed region, and the
whole-job throughput arithmetic.  No GPU and no nvidia-smi needed."""
import threading

import bench


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.thread = threading.Thread(target=lambda: None)
    s.thread.start()
    s.lines = list(lines)
    return s


def test_clock_summary_median_and_reasons():
    lines = [
        "2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1310.4, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "[N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = _sampler(lines).stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_hw_slowdown():
    lines = ["1500, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active"] * 4
    out = _sampler(lines).stop()
    assert out["sm_mhz"] == 1500.0
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_nvidia_smi():
    s = bench.ClockSampler(0)
    out = s.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_job_value_is_whole_job_over_slowest_rank():
    # 4 ranks x 1024 walkers x 10 steps in 2 s (the slowest rank) = 20480 evals/s
    assert bench.job_value(4, 1024, 10, 2000.0) == 20480.0
    assert bench.max_over_ranks(1, 3.5) == 3.5


def test_circular_statistics_of_the_sampler_angles():
    """Widths of phi_ref, lambda_L (period 2 pi) and psi_L (period pi) are taken on the
    circle: a cloud straddling the wrap has its own small width, not one of order pi."""
    import numpy as np

    rng = np.random.default_rng(0)
    c = 0.01 * rng.standard_normal((4000, 11))
    c[:, 5] = (0.02 * rng.standard_normal(4000)) % (2 * np.pi)
    c[:, 7] = (6.27 + 0.01 * rng.standard_normal(4000)) % (2 * np.pi)
    c[:, 9] = (3.13 + 0.02 * rng.standard_normal(4000)) % np.pi
    m, s = bench.circular_stats(c)
    assert abs(s[5] - 0.02) < 2e-3 and abs(s[7] - 0.01) < 1e-3 and abs(s[9] - 0.02) < 2e-3
    assert abs((m[7] - 6.27 + np.pi) % (2 * np.pi) - np.pi) < 1e-3
    assert abs((m[9] - 3.13 + np.pi / 2) % np.pi - np.pi / 2) < 2e-3
    assert abs(s[0] - 0.01) < 1e-3           # other coordinates as usual


def test_sky_mode_occupancy_bins():
    import numpy as np

    lam0 = 1.0
    c = np.zeros((8, 11))
    for k in range(8):
        c[k, 7] = (lam0 + (k % 4) * np.pi / 2 + 0.1) % (2 * np.pi)
        c[k, 8] = 0.3 if k < 4 else -0.3
    occ = bench.sky_mode_occupancy(c, lam0)
    assert np.allclose(occ, 1.0 / 8)
    assert abs(sum(bench.sky_mode_occupancy(c[:3], lam0)) - 1.0) < 1e-12


def test_sky_mode_lnl_per_mode():
    import numpy as np

    c = np.zeros((4, 11))
    c[:, 7] = [1.0, 1.0, 1.0 + np.pi, 1.0]
    c[:, 8] = [0.2, 0.2, 0.2, -0.2]
    out = bench.sky_mode_lnl(c, np.array([-3.0, -1.0, -50.0, -7.0]), 1.0)
    assert out[0] == [-1.0, -2.0] and out[2] == [-50.0, -50.0] and out[4] == [-7.0, -7.0]
    assert out[1] is None and out[3] is None
