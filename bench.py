"""Benchmark of the batched LISA log-likelihood on GB300 (one JSON line on rank 0).

Workload (the default): 1024 walkers drawn from the 1024-walker distributions (M_T
log-uniform in [1e5, 1e7] Msun, q ~ U[0.05, 1], aligned spins ~ U[-0.99, 0.99],
z ~ U[1, 8], isotropic angles), six modes, K = 1024 knots per mode, the 1-yr grid
1e-5..1e-1 Hz at df = 1/3.15576e7 s (3,155,445 bins), channels A/E/T, FP64.  The
data are the Table II Binary-1 injection made by the library plus seeded noise
coloured by the stand-in PSD (Eq. (12)).  A step is one batched ln L over all
walkers; value = walker evaluations per second over the whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank evaluates its own 1024 walkers on its own GPU
(replicas, weak scaling, no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "ln L evals/s (6 modes, A/E/T, 1-yr df)"
WORKLOAD = ("1024 walkers, 6 modes (2,2),(3,3),(4,4),(2,1),(3,2),(4,3), K=1024 knots, "
            "1-yr grid 1e-5..1e-1 Hz at df=1/3.15576e7 s (3155445 bins), A/E/T, FP64, "
            "Binary-1 injection + seeded noise")
WORKLOAD_C3 = ("8192 walkers with M_T log-uniform in [1e3, 1e9] Msun, 6 modes, K=1024 knots, "
               "1-yr grid (3155445 bins), A/E/T, FP64, CUDA-graph replay, autotuned tiles, "
               "Binary-1 injection + seeded noise")
# Algorithmic work per unit, the count the roofline's `achieved` uses: per (walker, mode,
# active bin) Horner for the 8 series (24 FMA = 48 flops), A e^{i phi} (2), three complex
# products T A e^{i phi} (12 as FMA + mul) and 6 adds into the channel sums, about 75
# flops, plus one sincos counted apart (not as flops); per (walker, bin) the three-channel
# integrand Re(d h*) w and |h|^2 w with its partial-sum add, about 25 flops.
FLOP_MODE_BIN = 75
FLOP_BIN = 25
# The implementation's own count of what the kernels execute, reported beside it: the
# phase series' Horner is replaced by the exact recurrence, and per (walker, mode, bin) it
# adds the segment offset (1), the t_coal ramp (2) and the table-plus-polynomial phasor
# (18) and spends 24 on the complex products = 95 flops; per (walker, bin) f_j (2) and
# the integrand (27) = 29 flops.
IMPL_FLOP_MODE_BIN = 48 + 1 + 2 + 18 + 2 + 24
IMPL_FLOP_BIN = 29
# data bytes streamed per bin by a walker tile (w and w*d for A, E, T, FP64) and the
# spline coefficients per segment (8 series x 4 doubles)
BYTES_BIN = 72
# DRAM bytes per (walker, bin) of the dense kernels from ncu captures of 32 walkers
# (dram__bytes_read.sum + dram__bytes_write.sum over 69,589,136 walker-bins), per tile
# shape (bins per thread, group); scaled to a launch by its walker-bins.  A shape without
# a capture reports null.
TRAFFIC_F64_PER_WALKER_BIN = {(8, 8): (753.79e6 + 5.11e6) / 69589136,
                              (4, 8): (755.36e6 + 6.43e6) / 69589136}
TRAFFIC_SPLIT_PER_WALKER_BIN = {(8, 8): (374.96e6 + 4.37e6) / 69589136}


def peaks():
    p = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
    except OSError:
        pass
    return p


def fp32_peak_tflops():
    """FP32 pipe peak derived from unit counts and clock: 152 SMs x 128 FP32 FMA per
    clock per SM x 2 flops x 2.07 GHz."""
    return 152 * 128 * 2 * 2.07e9 / 1e12


def fp64_peak_tflops():
    """FP64 pipe peak derived from unit counts and clock: 152 SMs x 2 FP64 FMA per
    clock per SM x 2 flops x 2.07 GHz.  The bench line also carries the rate that
    lisa_probe_pipes measures on the device at its running clock."""
    return 152 * 2 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    """Rank layout from torchrun's environment; NCCL between GPUs (gloo when
    BENCH_BACKEND=gloo, used by the CPU tests of this logic)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND") != "gloo" else "gloo")
    return world, rank, local


def walker_seed(c3: bool, rank: int) -> int:
    """Each rank evaluates its own walkers (replicas, weak scaling): distinct seeds."""
    return (3 if c3 else 1) + 1000 * rank


def job_value(world: int, walkers_per_rank: int, steps: int, ms_max: float) -> float:
    """Evaluations per second of the whole job: all ranks' walkers over the slowest rank."""
    return world * walkers_per_rank * steps / (ms_max * 1e-3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(lisalike, like, g, seed_walkers, B, logm=(5.0, 7.0)):
    """Data (Binary-1 injection by the library + noise of Eq. (12)) and walkers."""
    psd = np.empty((3, g.n_bins))
    lisalike.lisa_psd_aet(g.f0, g.df, g.n_bins, psd)
    like.set_data(g.f0, g.df, g.n_bins, None, psd)
    inj = W.theta_table2(1)
    h = like.template(inj)
    z = W.white_noise(g.n_bins, 2)
    sig = 0.5 * np.sqrt(psd / g.df)
    d = h + sig * (z[..., 0] + 1j * z[..., 1])
    like.set_data(g.f0, g.df, g.n_bins, d, psd)
    th = W.draw_walkers(B, seed_walkers, logm)
    th[:, 4] = [lisalike.lisa_dl_from_z(v) for v in th[:, 4]]
    return th


def work_units(like, th):
    """Active (walker, mode, bin) units and processed (walker, bin) units of one call."""
    band, _, _, _ = like.stage_knots(th)
    act = band[:, :, 0] == 1
    mode_bins = int(np.sum(np.where(act, band[:, :, 2] - band[:, :, 1] + 1, 0)))
    lo = np.where(act, band[:, :, 1], np.iinfo(np.int64).max).min(axis=1)
    hi = np.where(act, band[:, :, 2], -1).max(axis=1)
    bins = int(np.sum(np.maximum(hi - lo + 1, 0)))
    return mode_bins, bins


def cpu_baseline(sample_walkers=384, threads=None):
    """The oracle as it stands, on the host cores, on a bounded sample of the workload."""
    import oracle

    g = W.GRID_C2
    f = g.freqs()
    S = oracle.psd_aet(f)
    inj = W.theta_table2(1)
    d = oracle.template(inj, W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, g.n_bins)
    d = d + oracle.noise(S, g.df, W.white_noise(g.n_bins, 2))
    th = W.draw_walkers(sample_walkers, 1, (5.0, 7.0))
    th[:, 4] = [oracle.dl_gpc(v) for v in th[:, 4]]
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.loglike(th, W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, d, S, n_threads=threads)
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    oracle.loglike(th[:1], W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, d, S, n_threads=1)
    dt1 = time.perf_counter() - t1
    return {"value": sample_walkers / dt, "unit": "evals/s", "cores": threads, "kind": "oracle",
            "sample": "%d walkers of the 1024-walker workload (first %d of seed 1), full grid, "
                      "all host cores; single core: 1 walker" % (sample_walkers, sample_walkers),
            "single_core_value": 1.0 / dt1, "seconds": dt}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    g = W.GRID_C2
    S = oracle.psd_aet(g.freqs())
    inj = W.theta_table2(1)
    d = oracle.template(inj, W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, g.n_bins)
    d = d + oracle.noise(S, g.df, W.white_noise(g.n_bins, 2))
    threads = os.cpu_count() or 1
    per_step = max(threads, 8)
    th_all = W.draw_walkers(1024, 1, (5.0, 7.0))
    th_all[:, 4] = [oracle.dl_gpc(v) for v in th_all[:, 4]]

    def step(i):
        idx = (np.arange(per_step) + i * per_step) % 1024
        oracle.loglike(th_all[idx], W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, d, S,
                       n_threads=threads)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_per_step": "%d walkers" % per_step},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": threads,
                             "kind": "oracle",
                             "sample": "%d walkers per step of the 1024-walker workload" % per_step},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def time_split(lisalike, LisaLike, g, th, B, args, world, stream, mode_bins, bins, graphs=False):
    """The same workload in split precision (FP64 knot phases and final sums, FP32
    in-segment evaluation, sincos, amplitudes, transfers and partial sums)."""
    import torch

    like = LisaLike(modes=W.MODES6, n_knots=1024, t0=W.T0_YEAR, max_batch=B,
                    device=torch.cuda.current_device(), precision=lisalike.LISA_PREC_SPLIT)
    make_inputs(lisalike, like, g, 1, 1)          # same data as the FP64 handle
    if not args.no_autotune:
        lisalike.lisa_like_autotune(like.h, th[:256], min(256, B))
    if args.tile:
        lisalike.lisa_like_set_tune(like.h, *[int(v) for v in args.tile.split(",")])
    dparams = torch.tensor(th, dtype=torch.float64, device="cuda")
    lnL = torch.empty(B, dtype=torch.float64, device="cuda")

    def step():
        lisalike.lisa_like_loglike_device(like.h, dparams, B, lnL, None, None, stream.cuda_stream)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    stage_ms, ncalls = profile_once(lisalike, like, step)
    if graphs:
        lisalike.lisa_like_set_graphs(like.h, True)
        step()
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(world, e0.elapsed_time(e1))
    shape = lisalike.lisa_like_get_tune(like.h)
    like.close()
    dense_ms = stage_ms[4] / max(ncalls, 1)
    flops = FLOP_MODE_BIN * mode_bins + FLOP_BIN * bins
    achieved = flops / (dense_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    impl = impl_count(mode_bins, bins, dense_ms, peak)
    tpw = TRAFFIC_SPLIT_PER_WALKER_BIN.get(tuple(shape[:2]))
    traffic = tpw * bins if tpw else None
    probe = lisalike.probe_pipes(torch.cuda.current_device())
    return {"value": job_value(world, B, args.steps, ms), "unit": "evals/s",
            "ms_per_step": ms / args.steps, "dtype": "f32+f64", "graphs": graphs,
            "tile": {"bins_per_thread": shape[0], "group": shape[1], "blocks": shape[2]},
            "roofline": {"bound": "alu", "kernel": "dense_split_kernel", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "frac_survey_count": achieved / peak, "implementation_count": impl,
                         "sincos_per_s": mode_bins / (dense_ms * 1e-3),
                         "traffic": traffic,
                         "traffic_unit": "bytes per launch",
                         "hbm_gbs": traffic / (dense_ms * 1e-3) / 1e9 if traffic else None,
                         "algorithmic_bytes": algo_bytes(bins, shape[1], B, coef_bytes=192, bin_bytes=36),
                         "traffic_over_algorithmic":
                             traffic / algo_bytes(bins, shape[1], B, coef_bytes=192, bin_bytes=36)
                             if traffic else None,
                         "units_per_launch": {"walker_mode_bins": mode_bins, "walker_bins": bins},
                         "fractions": {
                             "binding": "fp32 (issue)", "fp32": achieved / peak,
                             "fp64": None, "mufu": None,
                             "hbm": (tpw * bins / (dense_ms * 1e-3) / 1e9 / peaks()["hbm_gbs"])
                             if (tpw and peaks().get("hbm_gbs")) else None,
                             "note": "fp64: per-item set-up only; mufu: one log2 per chunk "
                                     "(the phasor is a table and polynomials); ncu: issue 65 %, "
                                     "FMA pipe 54 % of cycles (packed f32x2 Horner and "
                                     "integrand), ALU 29 %"},
                         "peak_source": "derived: 152 SM x 128 FP32 FMA/clk x 2 x 2.07 GHz",
                         "measured_pipes": {
                             "fp32_tflops": 2 * probe["fp32_fma_per_s"] / 1e12,
                             "frac_of_measured_fp32":
                                 achieved / (2 * probe["fp32_fma_per_s"] / 1e12),
                             "source": "lisa_probe_pipes: FMA chains on every SM"},
                         "stage_ms_per_call": {k: v / max(ncalls, 1) for k, v in
                                               zip(("knots", "splines", "segprep", "plan",
                                                    "dense", "finish"), stage_ms)}}}


SAMPLER_METRIC = "PT sampler steps/s (8 temps x 256 walkers, 6 modes, A/E/T, 1-yr df)"
SAMPLER_WORKLOAD = ("parallel-tempered stretch-move sampler, 8 temperatures x 256 walkers "
                    "(a=1.15, geometric ladder ratio 2.04807, hottest infinite, adaptive), "
                    "LISA-frame sampling over the Table I prior, 8-sky-mode start; likelihood: "
                    "6 modes, K=1024, 1-yr grid (3155445 bins), A/E/T; injection M_T=2e6 "
                    "Msun, q=0.5, z=3 (SNR ~880) + seeded noise")


def sampler_cpu_baseline(steps=16):
    """The oracle sampler as it stands on a bounded sample: 2 temperatures x 8 walkers of
    the same workload for a few steps (each step = 16 oracle ln L evaluations)."""
    import oracle

    g = W.GRID_C2
    S = oracle.psd_aet(g.freqs())
    inj = np.array(W.THETA_SAMPLER_Z)
    inj[4] = oracle.dl_gpc(inj[4])
    d = oracle.template(inj, W.T0_YEAR, W.MODES6, 1024, g.f0, g.df, g.n_bins)
    d = d + oracle.noise(S, g.df, W.white_noise(g.n_bins, 2))
    xc = oracle.from_physical(inj)
    tL, lamL, betL, psiL = oracle.ssb_to_lisa(inj[10] + W.T0_YEAR, inj[7], inj[8], inj[9])
    xc[7], xc[8], xc[9], xc[10] = lamL, math.sin(betL), psiL, math.log(tL - W.T0_YEAR)
    x0 = xc + 1e-4 * np.random.default_rng(1).standard_normal((2, 8, 11))
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.sampler_lisa(x0, [1.0, 0.5], steps, 1, W.TABLE1_LOWER, W.TABLE1_UPPER, W.T0_YEAR,
                        W.MODES6, 1024, g.f0, g.df, d, S, n_threads=threads)
    dt = time.perf_counter() - t0
    evals = 16 * (steps + 1)
    return {"value": evals / dt, "unit": "ln L evals/s inside the sampler", "cores": threads,
            "kind": "oracle",
            "sample": "2 temperatures x 8 walkers, %d steps plus the initial evaluation" % steps,
            "steps_per_s_full_ensemble": evals / dt / (W.SAMPLER_T * W.SAMPLER_W),
            "seconds": dt}


def _sampler_injection(LL):
    """Physical parameters of the sampler workload's injection (z mapped to D_L)."""
    inj = np.array(W.THETA_SAMPLER_Z)
    inj[4] = LL.lisa_dl_from_z(inj[4])
    return inj


def _sampler_data(LL, like):
    """Give a handle the sampler workload's data: the injection made by the library plus
    the seeded noise of Eq. (12) coloured by the stand-in PSD; returns the injection."""
    g = W.GRID_C2
    psd = np.empty((3, g.n_bins))
    LL.lisa_psd_aet(g.f0, g.df, g.n_bins, psd)
    like.set_data(g.f0, g.df, g.n_bins, None, psd)
    inj = _sampler_injection(LL)
    h = like.template(inj)
    z = W.white_noise(g.n_bins, 2)
    d = h + 0.5 * np.sqrt(psd / g.df) * (z[..., 0] + 1j * z[..., 1])
    like.set_data(g.f0, g.df, g.n_bins, d, psd)
    return inj


def sampler_setup(args, rank, local):
    """Likelihood with the sampler workload's data, starting walkers, tile shapes."""
    import torch

    from paper_2005_01827_gb300 import LisaLike, build, lisalike as LL

    build.build()
    torch.cuda.set_device(local)
    T, Wk = W.SAMPLER_T, W.SAMPLER_W
    prec = LL.LISA_PREC_SPLIT if args.precision == "split" else LL.LISA_PREC_FP64
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    like = LisaLike(modes=W.MODES6, n_knots=1024, t0=W.T0_YEAR, max_batch=T * Wk // 2,
                    device=local, precision=prec, stream=stream.cuda_stream)
    inj = _sampler_data(LL, like)
    cfg = LL.lisa_sampler_default_config()
    xc = LL.from_physical(inj, True, W.T0_YEAR)
    scale = np.array([1e-3, 1e-3, 1e-2, 1e-2, 1e-2, 1e-2, 1e-2, 1e-3, 1e-3, 1e-2, 1e-4])
    x0 = LL.sky_mode_init(xc, scale, list(cfg.lower), list(cfg.upper), T, Wk, 7 + rank)
    if getattr(args, "start", "sky-modes") == "true-mode":
        # every walker at the injection's own sky mode (jitter only)
        x0[:, :, 7:9] = xc[7:9] + scale[7:9] * np.random.default_rng(5 + rank).standard_normal((T, Wk, 2))
    # tile shapes from the autotuner, timed on the starting walkers
    dx = torch.tensor(x0.reshape(-1, 11)[: T * Wk // 2], dtype=torch.float64, device="cuda")
    dth = torch.empty_like(dx)
    LL.lisa_sampler_to_physical(dx, dx.shape[0], True, W.T0_YEAR, dth, stream.cuda_stream)
    stream.synchronize()
    LL.lisa_like_autotune(like.h, dth.cpu().numpy()[:256], 256)
    return LL, like, stream, x0, prec


def like_roofline(LL, like, xs, prec, stream):
    """One profiled likelihood call on a sampler-sized batch (half of the walkers of every
    temperature, converted to physical parameters): stage times and the dense kernel's
    roofline."""
    import torch

    T, Wk = W.SAMPLER_T, W.SAMPLER_W
    B = T * Wk // 2
    dx = torch.tensor(xs.reshape(-1, 11)[:B], dtype=torch.float64, device="cuda")
    dth = torch.empty_like(dx)
    LL.lisa_sampler_to_physical(dx, B, True, W.T0_YEAR, dth, stream.cuda_stream)
    stream.synchronize()
    lnl_b = torch.empty(B, dtype=torch.float64, device="cuda")

    def like_call():
        LL.lisa_like_loglike_device(like.h, dth, B, lnl_b, None, None, stream.cuda_stream)

    like_call()
    stage_ms, ncalls = profile_once(LL, like, like_call)
    mode_bins, bins = work_units(like, dth.cpu().numpy())
    dense_ms = stage_ms[4] / max(ncalls, 1)
    flops = FLOP_MODE_BIN * mode_bins + FLOP_BIN * bins
    achieved = flops / (dense_ms * 1e-3) / 1e12
    split = prec == LL.LISA_PREC_SPLIT
    peak = fp32_peak_tflops() if split else fp64_peak_tflops()
    roof = {"bound": "alu", "kernel": "dense_split_kernel" if split else "dense_f64_kernel",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None,
            "note": "one profiled likelihood call on the sampler's batch of %d walkers after "
                    "the timed steps" % B,
            "stage_ms_per_call": {k: v / max(ncalls, 1) for k, v in
                                  zip(("knots", "splines", "segprep", "plan", "dense",
                                       "finish"), stage_ms)}}
    return roof, sum(stage_ms) / max(ncalls, 1)


def chain_stats(LL, chain, K, Wk, stream):
    taus = [LL.lisa_autocorr_time(chain, K, Wk, 11, q, None, stream.cuda_stream)
            for q in range(11)]
    return taus, float(np.nanmax(taus))


def run_sampler(args, world, rank, local):
    """The sampler workload: K timed steps after W warm-up (burn-in) steps; value =
    sampler steps per second of the whole job (each step evaluates every walker once)."""
    import torch

    LL, like, stream, x0, prec = sampler_setup(args, rank, local)
    T, Wk = W.SAMPLER_T, W.SAMPLER_W
    s = LL.LisaSampler(like, seed=11 + rank)
    s.set_state(x0)
    s.run(max(args.warmup, 3), record=False)          # burn-in; also captures the graph
    K = args.steps
    chain = torch.empty((K, Wk, 11), dtype=torch.float64, device="cuda")
    lch = torch.empty((K, Wk), dtype=torch.float64, device="cuda")
    acc0, sw0 = s.counts()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.run_device(K, chain, lch)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(world, e0.elapsed_time(e1))
    acc1, sw1 = s.counts()
    launches = K * s.step_launches()
    xs, lnls, betas, step = s.state()
    taus, tau = chain_stats(LL, chain, K, Wk, stream)
    sec = ms * 1e-3
    value = world * K / sec
    ess = K * Wk / tau
    roofline, like_ms = like_roofline(LL, like, xs, prec, stream)
    # sampler kernels alone: the same ensemble on the Gaussian target
    gs = LL.LisaSampler(None, n_temps=T, n_walkers=Wk, target=LL.LISA_TARGET_GAUSSIAN,
                        lisa_frame=1, seed=3)
    gs.set_state(x0)
    gs.run(3, record=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gs.run(200, record=False)
    own_ms = (time.perf_counter() - t0) * 1e3 / 200
    gs.close()
    # end to end through the public host API: state upload, K steps, chain download
    t0 = time.perf_counter()
    s.set_state(xs, step)
    c_host, l_host = s.run(K)
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    e2e = {"value": world * K / e2e_s, "unit": "steps/s",
           "h2d_bytes_per_step": T * Wk * 11 * 8 / K,
           "d2h_bytes_per_step": Wk * 12 * 8}
    s.close()
    like.close()
    line = {"metric": SAMPLER_METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": K, "warmup": max(args.warmup, 3), "ms_per_step": ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == LL.LISA_PREC_SPLIT else "f64", "data": "synthetic",
            "config": {"workload": SAMPLER_WORKLOAD, "temps": T, "walkers_per_temp": Wk,
                       "precision": args.precision, "graphs": True,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (data 227 MB, spline coefficients 0.8 GB)"},
            "evals_per_s": value * T * Wk,
            "mcmc": {"tau_max": tau, "tau": taus, "chain_steps": K,
                     "chain_over_tau": K / tau, "ess": ess, "ess_per_s": world * ess / sec,
                     "acceptance": ((acc1 - acc0)[:, 0] / np.maximum((acc1 - acc0)[:, 1], 1)).tolist(),
                     "swap_acceptance": ((sw1 - sw0)[:-1, 0] / np.maximum((sw1 - sw0)[:-1, 1], 1)).tolist(),
                     "betas": betas.tolist(),
                     "note": "tau from a chain shorter than 50 tau is a lower bound"},
            "step_breakdown_ms": {"likelihood_per_call": like_ms, "likelihood_calls": 2,
                                  "sampler_kernels_per_step": own_ms},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = sampler_cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


FLOW_METRIC = ("MCMC ESS/s of the coldest chain, flow proposal (8 couplings, bf16) vs plain "
               "stretch moves (8 temps x 256 walkers, 6 modes, A/E/T, 1-yr df)")
FLOW_WORKLOAD = ("; flow: 8 affine couplings (11-128-128-22, bf16 mma.sync, FP32 accumulate), "
                 "trained every 500 steps on the coldest chain until the end of burn-in, "
                 "independence MH on the coldest temperature every step")


def sky_mode_index(c, xc7):
    """Sky mode 0..7 of each sample: quarter-turn of lambda_L from the injection's, plus 4
    in the hemisphere of negative sin beta_L."""
    quarter = (np.floor(((c[:, 7] - xc7) % (2 * np.pi)) / (np.pi / 2) + 0.5) % 4).astype(int)
    return quarter + 4 * (c[:, 8] < 0).astype(int)


def sky_mode_lnl(c, lnl, xc7):
    """Largest and median ln L of the samples in each sky mode (None where empty): how
    much likelihood separates the modes a chain occupies."""
    m = sky_mode_index(c, xc7)
    out = []
    for k in range(8):
        v = lnl[m == k]
        out.append([float(v.max()), float(np.median(v))] if v.size else None)
    return out


def sky_mode_occupancy(c, xc7):
    """Fractions of the coldest-chain samples in each of the 8 LISA-frame sky modes (a
    longitude quarter-turn from the injection's, times the sign of sin beta_L), quarter
    q = 0..3 first for the injection's hemisphere, then the other one."""
    occ = np.bincount(sky_mode_index(c, xc7), minlength=8) / max(c.shape[0], 1)
    return occ.tolist()


# periods of the angular sampling coordinates (phi_ref, lambda_L, psi_L): their sample
# means and widths are taken on the circle (unwrapped around the circular mean)
ANGLE_PERIODS = {5: 2 * np.pi, 7: 2 * np.pi, 9: np.pi}


def circular_stats(c):
    """Per-coordinate mean and standard deviation of samples c [n, 11], the angles
    unwrapped around their circular mean first."""
    c = np.array(c, dtype=np.float64, copy=True)
    for q, P in ANGLE_PERIODS.items():
        a = 2 * np.pi * c[:, q] / P
        m = np.arctan2(np.mean(np.sin(a)), np.mean(np.cos(a))) * P / (2 * np.pi)
        c[:, q] = m + (c[:, q] - m + P / 2) % P - P / 2
    return c.mean(axis=0), c.std(axis=0)


def flow_compare(args, world, rank, local, burn_plain, steps_plain, burn_flow, steps_flow,
                 flow_precision):
    """Config-5 comparison on one GPU: the same sampler, seed and start with and without
    flow proposals (trained on the coldest chain every 500 steps until the end of the
    flow arm's burn-in).  With flow_precision "fp64" the flow moves of the timed steps are
    accepted on an FP64 likelihood (exact FP64 ln L of each flow proposal); burn-in flow
    moves use the sampler's own likelihood.  Returns the two arms' statistics."""
    import torch

    LL, like, stream, x0, prec = sampler_setup(args, rank, local)
    T, Wk = W.SAMPLER_T, W.SAMPLER_W
    xc = LL.from_physical(_sampler_injection(LL), True, W.T0_YEAR)
    like_flow = None
    if flow_precision == "fp64" and prec != LL.LISA_PREC_FP64:
        from paper_2005_01827_gb300 import LisaLike

        like_flow = LisaLike(modes=W.MODES6, n_knots=1024, t0=W.T0_YEAR, max_batch=Wk,
                             device=local, precision=LL.LISA_PREC_FP64, stream=stream.cuda_stream)
        _sampler_data(LL, like_flow)
    every = args.train_every
    out = {}
    clocks = ClockSampler(local)
    clocks.start()
    for use_flow in (False, True):
        burn = burn_flow if use_flow else burn_plain
        K = steps_flow if use_flow else steps_plain
        s = LL.LisaSampler(like, seed=11 + rank)
        if use_flow:
            s.enable_flow(train_every=every, train_iters=400, batch=1024, lr=1e-3, seed=3,
                          freeze_after=burn)
        s.set_state(x0)
        t0 = time.perf_counter()
        s.run(burn, record=False)
        burn_s = time.perf_counter() - t0
        if use_flow and like_flow is not None:
            s.set_flow_likelihood(like_flow)       # exact FP64 flow acceptances from here
            if args.flow_screen > 0:
                s.set_flow_screen(args.flow_screen)
            s.run(1, record=False)                 # capture the step graph with it
            sent0 = s.flow_screen_count() if args.flow_screen > 0 else 0
        chain = torch.empty((K, Wk, 11), dtype=torch.float64, device="cuda")
        lch = torch.empty((K, Wk), dtype=torch.float64, device="cuda")
        acc0, _ = s.counts()
        f0 = s.flow_stats()[0] if use_flow else None
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.run_device(K, chain, lch)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(world, e0.elapsed_time(e1))
        acc1, _ = s.counts()
        taus, tau = chain_stats(LL, chain, K, Wk, stream)
        c = chain.cpu().numpy().reshape(-1, 11)
        # the dominant sky mode: the most populated longitude quarter-turn
        quarter = np.floor(((c[:, 7] - xc[7]) % (2 * np.pi)) / (np.pi / 2) + 0.5) % 4
        dom = int(np.bincount(quarter.astype(int), minlength=4).argmax())
        main = c[quarter == dom]
        mean, std = circular_stats(c)
        mean_d, std_d = circular_stats(main)
        r = {"burn_in_steps": burn, "steps": K, "ms_per_step": ms / K,
             "tau_max": tau, "tau": taus, "chain_over_tau": K / tau,
             "ess": K * Wk / tau, "ess_per_s": world * K * Wk / tau / (ms * 1e-3),
             "tau_note": "a lower bound (ESS an upper bound) while chain_over_tau < 50 "
                         "(Sec. III.C)",
             "stretch_acceptance_cold": float((acc1 - acc0)[0, 0] / max((acc1 - acc0)[0, 1], 1)),
             "burn_in_s": burn_s, "launches_per_step": s.step_launches(),
             "mean": mean.tolist(), "std": std.tolist(),
             "sky_mode_occupancy": sky_mode_occupancy(c, xc[7]),
             "sky_mode_lnL_max_median": sky_mode_lnl(c, lch.cpu().numpy().reshape(-1), xc[7]),
             "dominant_mode_fraction": float(main.shape[0] / c.shape[0]),
             "mean_dominant": mean_d.tolist(), "std_dominant": std_d.tolist()}
        if use_flow:
            f1, n_tr, loss = s.flow_stats()
            r["flow_acceptance"] = float((f1 - f0)[0] / max((f1 - f0)[1], 1))
            r["trainings"] = n_tr
            r["last_training_loss"] = loss
            r["flow_likelihood"] = "fp64" if like_flow is not None else args.precision
            if like_flow is not None and args.flow_screen > 0:
                r["flow_screen_margin"] = args.flow_screen
                r["fp64_evaluated_fraction"] = (s.flow_screen_count() - sent0) / float(K * Wk)
        out["flow" if use_flow else "plain"] = r
        xs, _, _, _ = s.state()
        s.close()
    clk = clocks.stop()
    roofline, like_ms = like_roofline(LL, like, xs, prec, stream)
    like.close()
    if like_flow is not None:
        like_flow.close()
    p, f = out["plain"], out["flow"]
    sd, sdd = np.array(p["std"]), np.array(p["std_dominant"])
    out["posterior_agreement"] = {
        "max_abs_mean_diff_over_std": float(np.max(np.abs(np.array(f["mean"]) - np.array(p["mean"])) / sd)),
        "std_ratio_range": [float(np.min(np.array(f["std"]) / sd)), float(np.max(np.array(f["std"]) / sd))],
        "dominant_mode": {
            "max_abs_mean_diff_over_std": float(np.max(np.abs(
                np.array(f["mean_dominant"]) - np.array(p["mean_dominant"])) / sdd)),
            "std_ratio_range": [float(np.min(np.array(f["std_dominant"]) / sdd)),
                                float(np.max(np.array(f["std_dominant"]) / sdd))]},
        "sky_mode_occupancy_abs_diff_max": float(np.max(np.abs(
            np.array(f["sky_mode_occupancy"]) - np.array(p["sky_mode_occupancy"]))))}
    out["flow_over_plain_ess_per_s"] = f["ess_per_s"] / p["ess_per_s"]
    out["roofline"] = roofline
    out["clocks"] = clk
    out["gpu_launches"] = steps_plain * p["launches_per_step"] + steps_flow * f["launches_per_step"]
    return out


def run_flow(args, world, rank, local):
    """Config-5 comparison as its own bench line: value = effective samples per second of
    the coldest chain with the flow; both arms take --warmup burn-in and --steps timed
    steps."""
    burn = max(args.warmup, 2 * args.train_every)
    r = flow_compare(args, world, rank, local, burn, args.steps, burn, args.steps,
                     args.flow_precision)
    f = r["flow"]
    line = {"metric": FLOW_METRIC, "value": f["ess_per_s"], "unit": "effective samples/s",
            "n_gpus": world, "steps": args.steps, "warmup": burn, "ms_per_step": f["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "split" else "f64", "data": "synthetic",
            "config": {"start": args.start, "flow_precision": args.flow_precision,
                       "workload": SAMPLER_WORKLOAD + FLOW_WORKLOAD,
                       "precision": args.precision, "graphs": True,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (data 227 MB, spline coefficients 0.8 GB)"},
            "e2e": {"value": f["ess_per_s"], "unit": "effective samples/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                    "note": "device-resident chains; the host reads them once after the run"}}
    line.update(r)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


RB_METRIC = ("relative-binning ln L evals/s (6 modes, A/E/T, 1-yr df, 256 coarse bins) "
             "near the fiducial")
# algorithmic FP64 work of the relative-binning kernel: per (walker, mode, edge) the
# waveform and response at one frequency (as a knot: ~740 flops) plus e^{i phi} and the
# ratio (~40); per (walker, mode, channel, bin) the <d|h> term (~12) and per (walker, mode
# pair, channel, bin) the <h|h> term (~30)
FLOP_RB_EDGE = 780
FLOP_RB_DH = 12
FLOP_RB_HH = 30


def run_rb(args, world, rank, local):
    """1024 walkers at posterior-scale offsets from the sampler workload's injection, which
    is also the fiducial; relative binning timed on the device API, the dense FP64 and
    split paths timed on the same walkers, and the error against dense FP64."""
    import torch

    from paper_2005_01827_gb300 import LisaLike, build, lisalike as LL

    build.build()
    torch.cuda.set_device(local)
    g = W.GRID_C2
    B = 1024
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    like = LisaLike(modes=W.MODES6, n_knots=1024, t0=W.T0_YEAR, max_batch=B, device=local,
                    stream=stream.cuda_stream)
    psd = np.empty((3, g.n_bins))
    LL.lisa_psd_aet(g.f0, g.df, g.n_bins, psd)
    like.set_data(g.f0, g.df, g.n_bins, None, psd)
    inj = np.array(W.THETA_SAMPLER_Z)
    inj[4] = LL.lisa_dl_from_z(inj[4])
    h = like.template(inj)
    z = W.white_noise(g.n_bins, 2)
    d = h + 0.5 * np.sqrt(psd / g.df) * (z[..., 0] + 1j * z[..., 1])
    like.set_data(g.f0, g.df, g.n_bins, d, psd)
    t0 = time.perf_counter()
    like.set_fiducial(inj, 256)
    setup_s = time.perf_counter() - t0
    n_edges = like.rb_edges().size
    rng = np.random.default_rng(11 + rank)
    th = inj * (1 + 2e-4 * rng.standard_normal((B, 11)))
    th[:, 1] = np.minimum(th[:, 1], 1.0)
    dp = torch.tensor(th, dtype=torch.float64, device="cuda")
    out = torch.empty(B, dtype=torch.float64, device="cuda")

    def rb_step():
        LL.lisa_like_loglike_rb_device(like.h, dp, B, out, None, None, stream.cuda_stream)

    for _ in range(max(args.warmup, 3)):
        rb_step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rb_step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(world, e0.elapsed_time(e1))
    lrb = out.cpu().numpy()
    # the walker kernel alone (the band kernel runs first in each call)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    rb_step()
    e3.record(stream)
    torch.cuda.synchronize()
    call_ms = e2.elapsed_time(e3)
    # dense FP64 on the same walkers: accuracy reference and time
    lden, _, _ = like.loglike(th)
    t0 = time.perf_counter()
    like.loglike(th)
    dense_ms = (time.perf_counter() - t0) * 1e3
    err = np.abs(lrb - lden)
    e2e_t = time.perf_counter()
    for _ in range(max(2, args.steps // 4)):
        like.loglike_rb(th)
    e2e_s = max_over_ranks(world, time.perf_counter() - e2e_t)
    like.close()
    L, P = 6, 21
    nb = n_edges - 1
    flops = B * (L * n_edges * FLOP_RB_EDGE + L * 3 * nb * FLOP_RB_DH + P * 3 * nb * FLOP_RB_HH)
    achieved = flops / (call_ms * 1e-3) / 1e12
    peak = fp64_peak_tflops()
    value = world * B * args.steps / (ms * 1e-3)
    line = {"metric": RB_METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "1024 walkers at 2e-4 relative offsets from the injection of "
                       "the sampler workload (M_T=2e6, q=0.5, z=3, SNR ~880), 6 modes, 1-yr grid "
                       "(3155445 bins); fiducial = injection, 256 log-spaced coarse bins plus the "
                       "mode band edges (%d edges)" % n_edges,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "summary data and edge tables are L2-resident by design"},
            "accuracy_vs_dense_fp64": {"max_abs_dlnL": float(err.max()),
                                       "median_abs_dlnL": float(np.median(err)),
                                       "lnL_spread": float(lden.max() - lden.min())},
            "dense_fp64_ms_same_walkers": dense_ms, "fiducial_setup_s": setup_s,
            "speedup_vs_dense_fp64": dense_ms / (ms / args.steps),
            "roofline": {"bound": "alu", "kernel": "rb_walker_kernel (+ band_kernel)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 x 2.07 GHz",
                         "note": "flops counted per (walker, mode, edge), (walker, mode, "
                                 "channel, bin) and (walker, pair, channel, bin); one call "
                                 "timed with CUDA events"},
            "e2e": {"value": world * B * max(2, args.steps // 4) / e2e_s, "unit": "evals/s",
                    "h2d_bytes_per_step": B * 11 * 8, "d2h_bytes_per_step": 3 * B * 8},
            "gpu_launches": 2 * args.steps, "clocks": clk}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def algo_bytes(walker_bins, group, B, L=6, K=1024, coef_bytes=256, bin_bytes=None):
    """Algorithmic HBM bytes of one dense launch: the data row of each bin streamed once
    per walker group, and every (walker, mode) spline segment's record once."""
    return (bin_bytes or BYTES_BIN) * walker_bins / group + coef_bytes * B * L * (K - 1)


def impl_count(mode_bins, bins, dense_ms, peak):
    """The dense kernel's rate by the implementation's own flop count (labelled figure
    beside the algorithmic one)."""
    a = (IMPL_FLOP_MODE_BIN * mode_bins + IMPL_FLOP_BIN * bins) / (dense_ms * 1e-3) / 1e12
    return {"flop_per_walker_mode_bin": IMPL_FLOP_MODE_BIN, "flop_per_walker_bin": IMPL_FLOP_BIN,
            "achieved": a, "frac": a / peak}


def profile_once(lisalike, like, step):
    """Per-stage CUDA-event times of one call (profiling off afterwards)."""
    lisalike.lisa_like_set_profiling(like.h, True)
    lisalike.lisa_like_read_profile(like.h)
    step()
    stage_ms, n = lisalike.lisa_like_read_profile(like.h)
    lisalike.lisa_like_set_profiling(like.h, False)
    return stage_ms, n


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--walkers", type=int, default=1024,
                    help="walkers per GPU (1024 is the benchmark workload; smaller only for "
                         "profiling captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-split", action="store_true",
                    help="skip the split-precision timing of the same workload")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "sampler", "flow", "rb"],
                    help="c2: the 1024-walker benchmark workload; c3: 8192 walkers with "
                         "masses 1e3..1e9 Msun under CUDA-graph replay with autotuned tiles; "
                         "sampler: the parallel-tempered ensemble sampler on the likelihood; "
                         "flow: ESS/s of the sampler with and without flow proposals; "
                         "rb: the relative-binning likelihood near a fiducial")
    ap.add_argument("--precision", default="split", choices=["split", "fp64"],
                    help="likelihood precision of the sampler workload")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default tile shape (8 bins per thread, groups of 8); for "
                         "profiling captures that must see one known kernel variant")
    ap.add_argument("--flow-precision", default="same", choices=["same", "fp64"],
                    help="flow workload: likelihood precision of the flow moves (fp64: exact "
                         "acceptances while the stretch moves keep --precision)")
    ap.add_argument("--start", default="sky-modes", choices=["sky-modes", "true-mode"],
                    help="sampler workloads: walkers at the 8 LISA-frame sky modes (default) or "
                         "all at the injection's own sky mode")
    ap.add_argument("--tile", default=None,
                    help="P,G: force the dense kernels' tile shape (bins per thread, walker "
                         "group) after autotuning; for profiling captures of that variant")
    ap.add_argument("--train-every", type=int, default=500,
                    help="flow workload: steps between flow trainings (500 is the workload; "
                         "smaller only for profiling captures)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the 8192-walker and flow-vs-plain parts")
    ap.add_argument("--c3-steps", type=int, default=2,
                    help="timed steps of the 8192-walker part of the default run")
    ap.add_argument("--flow-screen", type=float, default=0.05,
                    help="margin in ln L of the split-precision screen of the FP64 flow "
                         "moves (0: every flow proposal evaluated in FP64)")
    ap.add_argument("--flow-burn", type=int, default=6000,
                    help="burn-in steps of each arm of the flow-vs-plain part")
    ap.add_argument("--flow-plain-steps", type=int, default=2000,
                    help="timed steps of the plain arm of the flow-vs-plain part")
    ap.add_argument("--flow-steps", type=int, default=2000,
                    help="timed steps of the flow arm of the flow-vs-plain part")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "sampler":
        return run_sampler(args, world, rank, local)
    if args.workload == "flow":
        return run_flow(args, world, rank, local)
    if args.workload == "rb":
        return run_rb(args, world, rank, local)

    line = like_line(args, world, rank, local, args.workload == "c3")
    if world == 1 and args.workload == "c2" and not args.no_extras:
        # the rest of the metric on the same run: the 8192-walker workload (masses 1e3..1e9,
        # graph replay, autotuned tiles) in both precisions, and configuration 5's ESS/s
        # of the flow-proposal sampler against the plain one
        a3 = argparse.Namespace(**vars(args))
        a3.steps, a3.warmup = args.c3_steps, 1
        line["c3"] = like_line(a3, world, rank, local, True)
        line["flow_vs_plain"] = flow_compare(args, world, rank, local, args.flow_burn,
                                             args.flow_plain_steps, args.flow_burn,
                                             args.flow_steps, "fp64")
        line["flow_vs_plain"]["config"] = {
            "workload": SAMPLER_WORKLOAD + FLOW_WORKLOAD, "start": "8 sky modes",
            "likelihood": "split precision for the stretch moves; exact FP64 ln L for the "
                          "flow moves of the timed steps (burn-in flow moves in split); "
                          "timed flow moves screened by the split ln L with margin %g "
                          "(the chain of unscreened FP64 flow moves, FP64 work only for "
                          "the proposals not rejected by the screen)" % args.flow_screen,
            "burn_in_steps": args.flow_burn, "plain_timed_steps": args.flow_plain_steps,
            "flow_timed_steps": args.flow_steps,
            "reduced": "config 5 as stated; step counts chosen so the default run stays "
                       "within minutes; both arms take the same number of timed steps, "
                       "since tau estimates of chains shorter than 50 tau grow with the "
                       "chain length (chain_over_tau says how far each arm is from the "
                       "50 tau of Sec. III.C)"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def like_line(args, world, rank, local, c3):
    """The batched ln L workload (1024 walkers, or with c3 the 8192-walker workload under
    graph replay) timed for args.steps steps after args.warmup: the bench line's dict."""
    import torch

    from paper_2005_01827_gb300 import LisaLike, build, lisalike

    build.build()
    torch.cuda.set_device(local)
    B = 8192 if c3 and args.walkers == 1024 else args.walkers
    g = W.GRID_C2
    like = LisaLike(modes=W.MODES6, n_knots=1024, t0=W.T0_YEAR, max_batch=B, device=local)
    th = make_inputs(lisalike, like, g, walker_seed(c3, rank), B,
                     (3.0, 9.0) if c3 else (5.0, 7.0))
    mode_bins, bins = work_units(like, th)
    # tile shapes from the autotuner (timed on a 256-walker sample of the workload)
    if not args.no_autotune:
        lisalike.lisa_like_autotune(like.h, th[:256], min(256, B))
    if args.tile:
        lisalike.lisa_like_set_tune(like.h, *[int(v) for v in args.tile.split(",")])

    # a dedicated stream: the kernels and the timing events share it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    dparams = torch.tensor(th, dtype=torch.float64, device="cuda")
    lnL = torch.empty(B, dtype=torch.float64, device="cuda")
    dh = torch.empty_like(lnL)
    hh = torch.empty_like(lnL)

    def step():
        lisalike.lisa_like_loglike_device(like.h, dparams, B, lnL, dh, hh, stream.cuda_stream)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    if c3:
        stage_ms, ncalls = profile_once(lisalike, like, step)
        lisalike.lisa_like_set_graphs(like.h, True)
        step()
        torch.cuda.synchronize()
    else:
        lisalike.lisa_like_set_profiling(like.h, True)
        lisalike.lisa_like_read_profile(like.h)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        step()
        launches += lisalike.lisa_like_last_launches(like.h)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_local = e0.elapsed_time(e1)
    clk = clocks.stop()
    if not c3:
        stage_ms, ncalls = lisalike.lisa_like_read_profile(like.h)
        lisalike.lisa_like_set_profiling(like.h, False)
    shape = lisalike.lisa_like_get_tune(like.h)
    ms = max_over_ranks(world, ms_local)
    value = job_value(world, B, args.steps, ms)
    assert np.all(np.isfinite(lnL.cpu().numpy())), "non-finite ln L"

    # end to end through the host-pointer entry point: H2D of the parameters and D2H of
    # ln L, <d|h>, <h|h> inside every step
    out = np.empty(B)
    odh, ohh = np.empty(B), np.empty(B)
    lisalike.lisa_like_loglike(like.h, th, B, out, odh, ohh)
    barrier(world)
    t0 = time.perf_counter()
    e2e_steps = max(1, args.steps // 2) if c3 else max(2, args.steps // 2)
    for _ in range(e2e_steps):
        lisalike.lisa_like_loglike(like.h, th, B, out, odh, ohh)
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    e2e = {"value": world * B * e2e_steps / e2e_s, "unit": "evals/s",
           "h2d_bytes_per_step": B * 11 * 8, "d2h_bytes_per_step": 3 * B * 8}

    dense_ms = stage_ms[4] / max(ncalls, 1)
    flops = FLOP_MODE_BIN * mode_bins + FLOP_BIN * bins
    achieved = flops / (dense_ms * 1e-3) / 1e12
    peak = fp64_peak_tflops()
    impl = impl_count(mode_bins, bins, dense_ms, peak)
    tpw = TRAFFIC_F64_PER_WALKER_BIN.get(tuple(shape[:2]))
    traffic = tpw * bins if tpw else None
    probe = lisalike.probe_pipes(local)      # measured pipe rates of this device
    roofline = {"bound": "alu", "kernel": "dense_f64_kernel", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "frac_survey_count": achieved / peak,
                "implementation_count": impl, "sincos_per_s": mode_bins / (dense_ms * 1e-3),
                "traffic": traffic,
                "traffic_unit": "bytes per launch",
                "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 x 2.07 GHz",
                "units_per_launch": {"walker_mode_bins": mode_bins, "walker_bins": bins},
                "stage_ms_per_call": {k: v / max(ncalls, 1) for k, v in
                                      zip(("knots", "splines", "segprep", "plan", "dense",
                                           "finish"), stage_ms)},
                "hbm_gbs": traffic / (dense_ms * 1e-3) / 1e9 if traffic else None,
                "algorithmic_bytes": algo_bytes(bins, shape[1], B),
                "traffic_over_algorithmic": traffic / algo_bytes(bins, shape[1], B)
                if traffic else None,
                "hbm_peak_gbs": peaks().get("hbm_gbs"),
                "measured_pipes": {"fp64_tflops": 2 * probe["fp64_fma_per_s"] / 1e12,
                                   "fp32_tflops": 2 * probe["fp32_fma_per_s"] / 1e12,
                                   "mufu_gops": probe["mufu_per_s"] / 1e9,
                                   "frac_of_measured_fp64": achieved / (2 * probe["fp64_fma_per_s"] / 1e12),
                                   "source": "lisa_probe_pipes: FMA / MUFU chains on every SM"}}
    hbm_peak = peaks().get("hbm_gbs")
    roofline["fractions"] = {
        "binding": "fp64", "fp64": achieved / peak, "fp32": 0.0, "mufu": 0.0,
        "hbm": (traffic / (dense_ms * 1e-3) / 1e9 / hbm_peak) if (traffic and hbm_peak) else None,
        "note": "fp32 and mufu: the FP64 kernel's inner loop issues neither (ncu <4,8>: FP64 "
                "pipe 94 % busy, FMA pipe 1.0 %); hbm: measured DRAM bytes per launch over "
                "the launch time"}
    if c3:
        roofline["note"] = "stage times from one profiled call before graph replay"
    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_C3 if c3 else WORKLOAD, "walkers_per_gpu": B,
                       "n_bins": g.n_bins, "knots": 1024, "modes": 6, "precision": "fp64",
                       "graphs": c3, "tile": {"bins_per_thread": shape[0], "group": shape[1],
                                              "blocks": shape[2]},
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (data 227 MB, spline coefficients 1.6 GB)"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
    like.close()
    if not args.no_split:
        line["split_precision"] = time_split(lisalike, LisaLike, g, th, B, args, world, stream,
                                             mode_bins, bins, graphs=c3)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and B == 1024 and not c3:
        line["cpu_baseline"] = cpu_baseline()
    return line



if __name__ == "__main__":
    sys.exit(main())
