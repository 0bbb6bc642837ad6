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
# algorithmic work (see the design notes): per (walker, mode, active bin) 8 cubic Horner
# evaluations (48), the segment offset (1), the t_coal ramp (2), e^{i phi} (20: a table
# entry rotated by sine and cosine polynomials of the remaining angle), A e^{i phi} (2),
# three complex transfer products accumulated into the mode sum (24) = 97 flops; per
# (walker, bin) f_j (2) and the three-channel integrand (27) = 29 flops.
FLOP_MODE_BIN = 48 + 1 + 2 + 20 + 2 + 24
FLOP_BIN = 29
# data bytes streamed per bin by a walker tile (w and w*d for A, E, T, FP64) and the
# spline coefficients per segment (8 series x 4 doubles)
BYTES_BIN = 72
# DRAM bytes per (walker, bin) of dense_f64_kernel<8, 8> from one ncu capture of 32
# walkers (dram__bytes_read.sum + dram__bytes_write.sum = 751.3 MB over 69,589,136
# walker-bins); scaled to a launch by its walker-bins.  None once the kernel changes.
TRAFFIC_F64_PER_WALKER_BIN = 751.3e6 / 69589136


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
    clock per SM x 2 flops x 2.07 GHz (the unit count measured by an FMA-chain probe:
    1.19 TFLOP/s at the running clock)."""
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


def cpu_baseline(sample_walkers=16, threads=None):
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
    lisalike.lisa_like_autotune(like.h, th[:256], min(256, B))
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
    return {"value": job_value(world, B, args.steps, ms), "unit": "evals/s",
            "ms_per_step": ms / args.steps, "dtype": "f32+f64", "graphs": graphs,
            "tile": {"bins_per_thread": shape[0], "group": shape[1], "blocks": shape[2]},
            "roofline": {"bound": "alu", "kernel": "dense_split_kernel", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "peak_source": "derived: 152 SM x 128 FP32 FMA/clk x 2 x 2.07 GHz",
                         "stage_ms_per_call": {k: v / max(ncalls, 1) for k, v in
                                               zip(("knots", "splines", "segprep", "plan",
                                                    "dense", "finish"), stage_ms)}}}


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
    ap.add_argument("--workload", default="c2", choices=["c2", "c3"],
                    help="c2: the 1024-walker benchmark workload; c3: 8192 walkers with "
                         "masses 1e3..1e9 Msun under CUDA-graph replay with autotuned tiles")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch

    from paper_2005_01827_gb300 import LisaLike, build, lisalike

    build.build()
    torch.cuda.set_device(local)
    c3 = args.workload == "c3"
    B = 8192 if c3 and args.walkers == 1024 else args.walkers
    g = W.GRID_C2
    like = LisaLike(modes=W.MODES6, n_knots=1024, t0=W.T0_YEAR, max_batch=B, device=local)
    th = make_inputs(lisalike, like, g, walker_seed(c3, rank), B,
                     (3.0, 9.0) if c3 else (5.0, 7.0))
    mode_bins, bins = work_units(like, th)
    # tile shapes from the autotuner (timed on a 256-walker sample of the workload)
    lisalike.lisa_like_autotune(like.h, th[:256], min(256, B))

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
    traffic = TRAFFIC_F64_PER_WALKER_BIN * bins if shape[:2] == (8, 8) else None
    roofline = {"bound": "alu", "kernel": "dense_f64_kernel", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_unit": "bytes per launch",
                "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 x 2.07 GHz",
                "units_per_launch": {"walker_mode_bins": mode_bins, "walker_bins": bins},
                "stage_ms_per_call": {k: v / max(ncalls, 1) for k, v in
                                      zip(("knots", "splines", "segprep", "plan", "dense",
                                           "finish"), stage_ms)},
                "hbm_gbs": BYTES_BIN * bins / (dense_ms * 1e-3) / 1e9,
                "hbm_peak_gbs": peaks().get("hbm_gbs")}
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
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
