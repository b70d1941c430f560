"""Benchmark of the synchrotron ray march on GB300: LOS samples/s and maps+grad/s.

One step = one map + gradient evaluation of the JF12-type workload (Nside 64,
512 steps to 20 kpc, 408 MHz / 1.4 / 2.3 / 23 GHz, 16 free parameters): the
C-ABI call synax_adjoint in chi^2 mode, which marches every ray forward
(maps, chi^2 against a seeded target) and backwards (d chi^2 / d theta).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torch.distributed.run, one rank per GPU; every rank
evaluates its own map + gradient (independent parameter sets, as in an HMC
ensemble), no collective on the data path (weak scaling); rank 0 prints one
JSON line.  --impl reference times the FP64 CPU oracle (central finite
differences for the gradient) on the host cores instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LOS samples/s and maps+grad/s (Nside 64, 512 steps) at stated tolerance"
WORKLOAD = "JF12-type map+gradient, Nside 64, 512 steps, 4 freq, 16 params, chi^2 vs seeded target"

# Algorithmic operation model per LOS sample (the stated per-sample figure of
# the hot path: field model, emissivity, RM and four Faraday phases), FP32 ops
# counting FMA/ADD/MUL/compare as one, and MUFU (SFU) ops.  The adjoint step
# marches every sample forward once and backwards once with derivatives:
# three forward-equivalents.
FWD_FP32_OPS = 200
FWD_MUFU_OPS = 22
ADJ_FACTOR = 3
# The same count for every field model, without the Faraday phase: each
# frequency adds 8 FP32 operations (phase, reduction to one turn, complex
# accumulation) and 2 MUFU (sin, cos).  JF12-type: 168 + 14 (200 + 22 at four
# frequencies, as above).  WMAP-type (Eq. 12-13): 60 + 14, with the
# sqrt, reciprocal, exponentials, log and two sincos of the field.  Stacked
# (Eq. 16): 99 + 25, four sincos pairs.  Grid: 142 + 9, the trilinear
# blend and cell location in place of the field model; its adjoint adds 36
# FP32 of node weights and sums per sample.  The pipe whose share of the
# measured peaks (measure_peaks) is larger bounds each model.
# The MUFU operations split into two classes because their measured rates
# differ: 2^x (ex2) and the rest (lg2, sin, cos, rcp, rsqrt).  Of each
# model's field MUFU count the exponentials are: JF12-type 9 (two logistic
# transitions, halo and X-field profiles, the CR profile's two, n_e's two,
# the emissivity power), WMAP-type 6, stacked 5, grid 5 (e^{-2|z|}, the CR
# profile's two, n_e, the emissivity power).
MODEL_EX2 = {"jf12": 9, "wmap": 6, "wmap_stack": 5, "grid": 5}
FWD_EX2_OPS = 9
MODEL_OPS = {"jf12": (168, 14), "wmap": (60, 14), "wmap_stack": (99, 25), "grid": (142, 9)}
GRID_ADJ_EXTRA_FP32 = 36
# DRAM bytes (read + write) of one k_adjoint launch of this workload, from the
# ncu capture summarised in profiles/k_adjoint_jf12_nside64_512steps.md
ADJ_DRAM_BYTES = 2.438e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="synax", choices=["synax", "reference"])
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-set ensemble measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip timing the CPU oracle")
    ap.add_argument("--no-grid", action="store_true", help="skip the grid-model (Sec. 3.3) measurement")
    ap.add_argument("--only-grid", action="store_true",
                    help="run only the grid-model measurement (no interpolation study) and print its JSON")
    ap.add_argument("--grid-runs", type=int, default=10, help="timed steps of the grid-model measurement")
    ap.add_argument("--only-hmc", action="store_true", help="run only the HMC sampling measurement")
    ap.add_argument("--only-wmap-stack", action="store_true",
                    help="run only the stacked-WMAP (Eq. 16) measurement, --wmap-stack-runs timed steps")
    ap.add_argument("--wmap-stack-runs", type=int, default=10, help="timed steps of the stacked-WMAP measurement")
    ap.add_argument("--only-batch-low-res", action="store_true",
                    help="run only the 256-chain Nside-16 batch measurement and print its JSON (a profiling aid)")
    ap.add_argument("--no-surrogate", action="store_true", help="skip training and timing the learned surrogate")
    ap.add_argument("--surrogate-steps", type=int, default=20000, help="Adam steps of the surrogate training")
    ap.add_argument("--surrogate-maps", type=int, default=50000, help="training maps of the surrogate")
    ap.add_argument("--only-surrogate", action="store_true",
                    help="run only the surrogate section and print its object (a profiling aid)")
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 8, 16, 32],
                    help="lanes per ray for every launch (0: autotune per step-count bin)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smmax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smmax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smmax) if smmax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measure_peaks(sx) -> dict:
    """FP32 and SFU throughput measured on this GPU (synax_pipe_peak): the
    FP32 peak is the faster of scalar FFMA and paired FFMA2 (element
    operations); the SFU has two measured rates, ex2 and the slowest of the
    other instructions the march uses (lg2, sin, cos, rcp, rsqrt)."""
    r = sx.pipe_peaks(iters=16384)
    mufu = {k: r[k] / 1e12 for k in ("ex2", "lg2", "sin", "cos", "rcp", "rsqrt")}
    return {"fp32_top": max(r["ffma"], r["ffma2"]) / 1e12, "mufu_ex2": mufu["ex2"],
            "mufu_other": min(v for k, v in mufu.items() if k != "ex2"),
            "unit": "T element op/s", "ffma": r["ffma"] / 1e12, "ffma2": r["ffma2"] / 1e12, "mufu": mufu,
            "sfu_conversions": {"frnd": r["frnd"] / 1e12, "f2i": r["f2i"] / 1e12}, "sms": r["sms"]}


def roofline_alu(fp32_ops: float, mufu_ops: float, t_s: float, peaks: dict, kernel: str,
                 ex2_ops: float = 0.0) -> dict:
    """Roofline of a march kernel from its algorithmic FP32 and MUFU
    operations (ex2_ops of the MUFU ones are exponentials) over a measured
    duration t_s.  Each pipe's roofline time is its operations over its
    measured rates; the pipe with the longer roofline time bounds the kernel
    and frac = that time / t_s.  For MUFU, peak is the effective rate of the
    kernel's mix (mufu_ops over its roofline time)."""
    t_fp32 = fp32_ops / (peaks["fp32_top"] * 1e12)
    t_mufu = ex2_ops / (peaks["mufu_ex2"] * 1e12) + (mufu_ops - ex2_ops) / (peaks["mufu_other"] * 1e12)
    mufu_eff = mufu_ops / t_mufu / 1e12 if t_mufu > 0 else float("inf")
    if t_fp32 >= t_mufu:
        pipe, ach, peak, frac, other = "FP32", fp32_ops / t_s / 1e12, peaks["fp32_top"], t_fp32 / t_s, t_mufu / t_s
    else:
        pipe, ach, peak, frac, other = "MUFU", mufu_ops / t_s / 1e12, mufu_eff, t_mufu / t_s, t_fp32 / t_s
    return {"bound": "alu", "pipe": pipe, "achieved": ach, "peak": peak, "unit": f"T {pipe} op/s",
            "frac": frac, "frac_other_pipe": other, "kernel": kernel,
            "peak_basis": f"measured peaks of this GPU (synax_pipe_peak, peaks_measured; "
                          f"{'max of FFMA, FFMA2' if pipe == 'FP32' else 'ex2 and other-SFU rates weighted by the mix'})"}


def march_roofline(model: str, n_freq: int, samples_per_s: float, peaks: dict, adjoint: bool,
                   kernel: str) -> dict:
    """Roofline of a march kernel from the per-sample operation counts of
    MODEL_OPS against the measured pipe peaks."""
    fp32, mufu = MODEL_OPS[model]
    ex2 = MODEL_EX2[model]
    fp32 += 8 * n_freq
    mufu += 2 * n_freq
    if adjoint:
        fp32 = ADJ_FACTOR * fp32 + (GRID_ADJ_EXTRA_FP32 if model == "grid" else 0)
        mufu = ADJ_FACTOR * mufu
        ex2 = ADJ_FACTOR * ex2
    out = roofline_alu(samples_per_s * fp32, samples_per_s * mufu, 1.0, peaks, kernel, samples_per_s * ex2)
    out["ops_per_sample"] = {"fp32": fp32, "mufu": mufu, "mufu_ex2": ex2}
    return out


def oracle_row(prob, n_pix_sample: int, free, note: str = "") -> dict:
    """The FP64 oracle on a pixel sample of a workload: one map and
    central differences over the parameters `free` (2 maps each); LOS samples
    of the map + gradient per second of host time."""
    import oracle
    from paper_2410_01136_gb300 import inputs
    oracle.build()
    pix = inputs.sample_pixels(prob.npix, n_pix_sample, seed=41)
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    oracle.forward(prob, pix=pix, threads=threads)
    for i in free:
        for sgn in (1.0, -1.0):
            th = prob.theta.copy()
            th[i] += sgn * 1e-4 * max(abs(th[i]), 1e-3)
            oracle.forward(prob.with_theta(th), pix=pix, threads=threads)
    dt = time.perf_counter() - t0
    rate = pix.size * prob.n_steps / dt
    out = {"samples_per_s": rate, "maps_grad_per_s": rate / prob.samples, "cores": threads, "seconds": dt,
           "kind": "oracle", "sample": f"{pix.size} of {prob.npix} pixels x {prob.n_steps} steps, map + "
                                       f"{2 * len(free)}-map central-difference gradient"}
    if note:
        out["note"] = note
    return out


def slowest_rank_times(times, device=None) -> list:
    """Each per-rank time (ms) replaced by its maximum over the ranks of the
    initialised process group (the job takes as long as its slowest rank);
    unchanged on one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(x) for x in times]
    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(world: int, units_per_rank: float, ms: float) -> float:
    """Units of all ranks over the slowest rank's time (weak scaling: every
    rank processes its own units)."""
    return world * units_per_rank / (ms * 1e-3)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): FD gradient on a pixel sample
# ---------------------------------------------------------------------------
def oracle_map_grad_rate(n_pix_sample: int, n_repeat: int = 1, threads: int | None = None
                         ) -> tuple[float, float, int, str]:
    """samples/s of map + gradient with the FP64 oracle: per map+grad, one
    forward and 2 * 16 central-difference maps, on n_pix_sample pixels, on
    `threads` host threads (default: every core)."""
    import numpy as np

    import oracle
    from paper_2410_01136_gb300 import inputs
    oracle.build()
    prob, _, _ = inputs.config3()
    pix = inputs.sample_pixels(prob.npix, n_pix_sample, seed=41)
    h = 1e-4 * inputs.jf12_scales(prob.theta)
    threads = threads or oracle.default_threads()
    t0 = time.perf_counter()
    for _ in range(n_repeat):
        oracle.forward(prob, pix=pix, threads=threads)
        for i in range(prob.theta.size):
            for sgn in (1.0, -1.0):
                th = prob.theta.copy()
                th[i] += sgn * h[i]
                oracle.forward(prob.with_theta(th), pix=pix, threads=threads)
    dt = time.perf_counter() - t0
    samples = n_repeat * pix.size * prob.n_steps        # LOS samples of the map+grad evaluations
    sample_desc = (f"{pix.size} of {prob.npix} pixels x {prob.n_steps} steps x 4 freq, "
                   f"map + 32-map central-difference gradient, {n_repeat} evaluation(s)")
    return samples / dt, dt, threads, sample_desc


def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo), or the platform string."""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    per_step = []
    rate = None
    threads = 1
    desc = ""
    n_pix = 1024          # ~0.7 s of host time per step on 16 cores
    for k in range(args.warmup + args.steps):
        r, dt, threads, desc = oracle_map_grad_rate(n_pix)
        if k >= args.warmup:
            per_step.append(dt)
            rate = r if rate is None else rate
    rates = [n_pix * 512 / d for d in per_step]
    value = float(np.mean(rates))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(per_step)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nside": 64, "n_steps": 512, "n_freq": 4,
                   "sample": f"{n_pix} pixels per step"},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def bench_batch(sx, inputs, torch, dev, n_runs: int = 3, sets=None, name=None) -> dict:
    """An ensemble of map+gradient evaluations: one persistent graph-captured
    launch per evaluation, against the same sets as one-map synax_adjoint
    calls in a row.  Default: the 256-set ensemble (Nside 16-128, 128-1024
    steps, theta ~ 5% around the fiducial)."""
    import numpy as np
    sets = inputs.config4() if sets is None else sets
    targets = []
    for i, p in enumerate(sets):
        t = sx.forward(p.with_theta(inputs.perturbed_theta(p.theta, seed=100 + i))).contiguous()
        targets.append(t)
    samples = sum(p.samples for p in sets)
    plan = sx.BatchPlan(sets)
    info = plan.info()
    stream = torch.cuda.current_stream(dev)
    grads, chi2 = plan.run(targets=targets, sigma=0.5)            # captures the graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_runs):
        plan.run(targets=targets, sigma=0.5, grads=grads, chi2=chi2)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1) / n_runs
    lat = plan.latencies()
    plan.close()
    # the same ensemble with every set marched alone (no two-set items)
    sx.set_batch_pairing(False)
    try:
        plan1 = sx.BatchPlan(sets)
        plan1.run(targets=targets, sigma=0.5, grads=grads, chi2=chi2)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n_runs):
            plan1.run(targets=targets, sigma=0.5, grads=grads, chi2=chi2)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_unpaired = e0.elapsed_time(e1) / n_runs
        plan1.close()
    finally:
        sx.set_batch_pairing(True)
    ws = torch.empty(max(sx.adjoint_workspace_bytes(p) for p in sets), dtype=torch.uint8, device=dev)
    for p, t in zip(sets[:4], targets[:4]):
        sx.adjoint(p, target=t, sigma=0.5, workspace=ws)
    torch.cuda.synchronize()
    e0.record(stream)
    for p, t in zip(sets, targets):
        sx.adjoint(p, target=t, sigma=0.5, workspace=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    return {
        "workload": name or "256 JF12-type sets, Nside {16..128} x steps {128..1024}, chi^2 map+gradient",
        "samples_per_run": samples,
        "ms_per_run": ms_batch,
        "samples_per_s": samples / (ms_batch * 1e-3),
        "maps_grad_per_s": len(sets) / (ms_batch * 1e-3),
        "latency_ms_p50": float(np.percentile(lat, 50)),
        "latency_ms_p99": float(np.percentile(lat, 99)),
        "sequential_ms": ms_seq,
        "sequential_maps_grad_per_s": len(sets) / (ms_seq * 1e-3),
        "speedup_vs_sequential": ms_seq / ms_batch,
        "unpaired_ms": ms_unpaired,
        "pairing_note": "the plan marches sets of one ray geometry two at a time, sharing their position-only "
                        "field work; unpaired_ms is the same ensemble with every set alone",
        "plan": info,
    }


def bench_grid(sx, inputs, torch, dev, n_runs: int = 10, n_fit: int = 50) -> dict:
    """The field-level workload (Sec. 3.3): B on 128 x 128 x 32 nodes over the
    (40, 40, 10) kpc box, Nside 64, 512 steps to the walls, Q/U at 2.4 GHz;
    one step = synax_adjoint_grid in chi^2 mode (maps, chi^2 against a mock
    from another seeded grid plus 1 mK noise, theta gradient and the
    1.57-million-value grid gradient).  L2 flushed between steps."""
    import numpy as np
    prob = inputs.grid_problem()
    grid = torch.tensor(np.asarray(prob.grid), dtype=torch.float32, device=dev)
    prob = prob.replace(grid=grid)
    mock = sx.forward(inputs.grid_problem(seed=22).replace(grid=torch.tensor(
        inputs.grid_field(seed=22), dtype=torch.float32, device=dev)))
    target = (mock + 1e-3 * torch.tensor(inputs.target_noise(tuple(mock.shape), seed=23, sigma=1.0),
                                         dtype=torch.float32, device=dev)).contiguous()
    maps = torch.empty_like(target)
    gg = torch.empty_like(grid)
    ws = torch.empty(max(sx.adjoint_grid_workspace_bytes(prob), 1), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        return sx.adjoint_grid(prob, target=target, sigma=1e-3, maps_out=maps, grid_grad=gg, workspace=ws)

    for _ in range(3):
        step()
        sx.forward(prob, out=maps)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_runs)]
    fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_runs)]
    for k in range(n_runs):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    for k in range(n_runs):
        flush.fill_(float(k))
        fev[k][0].record(stream)
        sx.forward(prob, out=maps)
        fev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    ms_fwd = float(np.mean([a.elapsed_time(b) for a, b in fev]))
    # the field-level fit of Sec. 3.3: chi^2 + grid gradient + Adam per step
    fit = sx.GridFit(prob, target, sigma=1e-3, lr=0.05)
    fit.run(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    chi2 = fit.run(n_fit)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fit = e0.elapsed_time(e1) / n_fit
    chi2 = chi2.cpu().numpy()
    samples = prob.samples
    return {
        "workload": "grid B 128x128x32 over (40, 40, 10) kpc, Nside 64, 512 steps to the box, 2.4 GHz, "
                    "chi^2 map + theta gradient + grid gradient",
        "samples_per_step": samples,
        "grid_values": int(grid.numel()),
        "ms_per_step": ms,
        "samples_per_s": samples / (ms * 1e-3),
        "maps_grad_per_s": 1.0 / (ms * 1e-3),
        "forward_ms": ms_fwd,
        "forward_samples_per_s": samples / (ms_fwd * 1e-3),
        "gpu_launches_per_step": 3,      # k_adjoint, k_reduce_partials, k_grid_unpad (plus a memset)
        "fit_ms_per_step": ms_fit,
        "fit_200_steps_s": 200 * ms_fit * 1e-3,
        "fit_chi2_first_last": [float(chi2[0]), float(chi2[-1])],
        "fit_steps_timed": n_fit,
        "fit_note": "Adam, lr 0.05 uG, on the grid (synax_adam), back to back without L2 flushes",
        "l2": "flushed between steps (256 MiB write); the 6.3 MB grid is re-read from HBM",
    }


def bench_wmap_stack(sx, inputs, torch, dev, n_runs: int = 10) -> dict:
    """Sec. 4.3's 16-parameter model: the stacked WMAP field of Eq. 16 in
    the (40, 40, 10) kpc box, Nside 64, 512 steps, I/Q/U at 2.4 GHz; one step
    = synax_adjoint in chi^2 mode (map + 19-component gradient: the 16 field
    parameters and N0_obs, p, n_e0) against a mock with 1 mK noise.  L2
    flushed between steps."""
    import numpy as np
    prob = inputs.wmap_stack_problem()
    th_mock = prob.theta * (1.0 + 0.03 * inputs.normal(inputs.substream(72, 1), prob.theta.size))
    mock = sx.forward(prob.with_theta(th_mock))
    target = (mock + 1e-3 * torch.tensor(inputs.target_noise(tuple(mock.shape), seed=73, sigma=1.0),
                                         dtype=torch.float32, device=dev)).contiguous()
    maps = torch.empty_like(target)
    ws = torch.empty(max(sx.adjoint_workspace_bytes(prob), 1), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        sx.adjoint(prob, target=target, sigma=1e-3, maps_out=maps, workspace=ws)
        sx.forward(prob, out=maps)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_runs)]
    fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_runs)]
    for k in range(n_runs):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        sx.adjoint(prob, target=target, sigma=1e-3, maps_out=maps, workspace=ws)
        ev[k][1].record(stream)
    for k in range(n_runs):
        flush.fill_(float(k))
        fev[k][0].record(stream)
        sx.forward(prob, out=maps)
        fev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    ms_fwd = float(np.mean([a.elapsed_time(b) for a, b in fev]))
    return {"workload": "stacked WMAP (Eq. 16), box (40, 40, 10) kpc, Nside 64, 512 steps, 2.4 GHz, "
                        "chi^2 map + 19-component gradient",
            "samples_per_step": prob.samples, "ms_per_step": ms, "maps_grad_per_s": 1.0 / (ms * 1e-3),
            "samples_per_s": prob.samples / (ms * 1e-3), "forward_ms": ms_fwd,
            "forward_samples_per_s": prob.samples / (ms_fwd * 1e-3), "gpu_launches_per_step": 2}


def hmc_problem(inputs):
    """The WMAP-type map of the sampling workload at the Sec. 3.1 values."""
    import numpy as np
    th = np.array([1.2, 0.4712, 0.0157, 0.4363, 0.0, inputs.N0_EARTH, 3.0, 0.03])
    return inputs.Problem(nside=64, n_steps=512, freq_hz=(2.4e9,), model_id=inputs.MODEL_WMAP, theta=th,
                          box_clip=True, obs_kpc=inputs.OBS_PAPER_KPC)


def bench_hmc(sx, inputs, torch, dev, n_chains: int = 16, n_warm: int = 40, n_draws: int = 60) -> dict:
    """Gradient-based sampling as in Sec. 3.2: the WMAP-type model with the
    Sec. 3.1 values (b0 = 1.2 uG, psi0 = 0.4712, psi1 = 0.0157, chi0B =
    0.4363; no x field; N0_obs, p, n_e0 fixed) in the (40, 40, 10) kpc box,
    Nside 64, 512 steps, 2.4 GHz, a mock with 1 mK noise; HMC chains on the
    batch (synax_hmc_*), the four field parameters free, diagonal Laplace
    mass, warm-up then timed draws; ESS per second of sampling over all
    chains (multi-chain ESS)."""
    import numpy as np
    prob = hmc_problem(inputs)
    th = prob.theta
    mock = sx.forward(prob)
    target = (mock + 1e-3 * torch.tensor(inputs.target_noise(tuple(mock.shape), seed=84, sigma=1.0),
                                         dtype=torch.float32, device=dev)).contiguous()
    free = [0, 1, 2, 3]
    inv_mass = sx.laplace_inv_mass(prob, target, 1e-3, free)
    sd = np.sqrt(inv_mass)
    th0 = np.stack([th + sd * inputs.normal(inputs.substream(85, c), th.size) for c in range(n_chains)])
    hmc = sx.HMC([prob.with_theta(t) for t in th0], [target] * n_chains, 1e-3, th0, step_size=0.5, n_leapfrog=8,
                 seed=86, inv_mass=inv_mass)
    hist = hmc.warmup(n_warm, adapt_mass=False)          # the Laplace mass already sets the scales
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    draws, acc = hmc.run(n_draws)
    e1.record(stream)
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) * 1e-3
    d = draws.cpu().numpy()
    ess = sx.effective_sample_size(d[:, :, free])
    post_sd = d[:, :, free].reshape(-1, len(free)).std(axis=0)
    hmc.close()
    return {"workload": "WMAP-type (Sec. 3.1 values), box (40, 40, 10) kpc, Nside 64, 512 steps, 2.4 GHz, sigma 1 mK; "
                        f"{n_chains} HMC chains x {n_draws} draws after {n_warm} warm-up, 8 leapfrog steps, "
                        "b0, psi0, psi1, chi0B free",
            "seconds_sampling": s, "ms_per_iteration": 1e3 * s / n_draws, "samples_per_map": prob.samples,
            "gradient_evals_per_s": n_chains * 8 * n_draws / s,
            "acceptance": float(acc.float().mean().item()),
            "final_step_size": hist[-1][0] if hist else None,
            "ess": {k: float(v) for k, v in zip(["b0", "psi0", "psi1", "chi0B"], ess)},
            "ess_per_s": {k: float(v / s) for k, v in zip(["b0", "psi0", "psi1", "chi0B"], ess)},
            "posterior_sd": {k: float(v) for k, v in zip(["b0", "psi0", "psi1", "chi0B"], post_sd)},
            "paper_context_ess_per_s_nuts_a100": {"b0": 1.90, "psi0": 1.73, "psi1": 1.07, "chi0B": 0.87}}


def interp_study(sx, inputs, torch) -> dict:
    """Sec. 5's interpolation study, re-run: the WMAP-type field with the
    parameters of Sec. 3.1 (b0 = 1.2 uG, psi0 = 0.4712, psi1 = 0.0157,
    chi0B = 0.4363 rad; no x field; analytic n_e) sampled on (N, N, N/4)
    grids over the (40, 40, 10) kpc box and marched as a grid model, against
    the analytic march: std over pixels of the I, Q, U residual (K) at
    2.4 GHz, Nside 64, 512 steps, FP64.  Reported, not timed."""
    import numpy as np
    th = np.array([1.2, 0.4712, 0.0157, 0.4363, 0.0, inputs.N0_EARTH, 3.0, 0.03])
    ana = inputs.Problem(nside=64, n_steps=512, freq_hz=(2.4e9,), model_id=inputs.MODEL_WMAP, theta=th,
                         box_clip=True, obs_kpc=inputs.OBS_PAPER_KPC, f64=True)
    m_ana = sx.forward(ana)
    out = {"workload": "WMAP-type (Sec. 3.1 values) on (N, N, N/4) grids vs analytic, Nside 64, 512 steps, "
                       "2.4 GHz, FP64", "std_IQU_K": {}, "map_rms_IQU_K": [float(x) for x in
                                                     m_ana[0].pow(2).mean(dim=-1).sqrt().tolist()]}
    for n_x in (64, 128, 256, 512):
        grid = sx.grid_sample(ana, (n_x, n_x, n_x // 4))
        pg = inputs.Problem(nside=64, n_steps=512, freq_hz=(2.4e9,), model_id=inputs.MODEL_GRID,
                            theta=np.array([th[5], th[6], th[7]]), box_clip=True, obs_kpc=inputs.OBS_PAPER_KPC,
                            f64=True, grid=grid)
        r = (sx.forward(pg) - m_ana)[0]
        out["std_IQU_K"][str(n_x)] = [float(x) for x in r.std(dim=-1).tolist()]
        del grid, pg, r
    torch.cuda.empty_cache()
    return out


def bench_surrogate_sh(sx, inputs, torch, dev, steps: int, n_maps: int = 50000) -> dict:
    """The surrogate on the low-order basis (the first 3072 real spherical
    harmonics, l <= 55): same network, data and training as bench_surrogate,
    judged on the 512 held-out draws as a full-map error: the in-subspace
    RMS of the judge combined with each true map's own truncation outside
    the basis (||x||^2 - ||c||^2 per Stokes map, over npix)."""
    import numpy as np
    from paper_2410_01136_gb300.surrogate import Surrogate
    prob = inputs.config5_problem()
    sur = Surrogate.for_workload(batch=512, total_steps=steps, lr=1e-3, lr_min=1e-5, basis="sh")
    thetas = inputs.config5_thetas(n_maps, seed=50)
    t0 = time.perf_counter()
    sur.dataset(prob, thetas)
    sur.train(steps, seed=1)
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t0
    hold = inputs.config5_thetas(512, seed=51)
    c = sur(torch.tensor(hold, dtype=torch.float32, device=dev))
    _, rms, _ = sur.judge(prob, hold, c, 1.0)
    rms = rms.cpu().numpy()
    npix = 12 * 64 * 64
    trunc = np.empty((512, 3))
    for k in range(0, 512, 64):
        maps = torch.stack([sx.forward(prob.with_theta(t))[0] for t in hold[k:k + 64]])      # [64, 3, npix]
        cc = sur.project(maps.reshape(-1, npix)).reshape(64, 3, -1).double()
        x2 = maps.double().pow(2).sum(dim=-1)
        trunc[k:k + 64] = ((x2 - cc.pow(2).sum(dim=-1)).clamp_min(0.0) / npix).sqrt().cpu().numpy()
    full = np.sqrt(rms.astype(np.float64) ** 2 + trunc ** 2)
    sur.close()

    def q(a):
        return {"median": float(np.median(a)), "p90": float(np.percentile(a, 90))}
    return {"workload": "as 'surrogate', basis = real spherical harmonics l <= 55 (first 3072), orthonormalised",
            "dataset_and_train_s": t_all,
            "in_subspace_rms_K": {n: q(rms[:, i]) for i, n in enumerate("IQU")},
            "truncation_rms_K": {n: q(trunc[:, i]) for i, n in enumerate("IQU")},
            "full_map_rms_K": {n: q(full[:, i]) for i, n in enumerate("IQU")},
            "pass_frac_1K_full_map_I": float(np.mean(full[:, 0] <= 1.0)),
            "pass_frac_1K_full_map_all": float(np.mean(full.max(axis=1) <= 1.0))}


def bench_surrogate(sx, inputs, torch, dev, steps: int, peaks: dict, n_maps: int = 50000) -> dict:
    """The learned surrogate on its workload: 50 000 Nside-64 JF12-type maps at
    408 MHz (parameters uniform in +-20 % of the fiducial scale), an MLP
    16 -> 1024 x 4 -> 3 x 3072, judged by the march on 512 held-out draws."""
    import numpy as np
    from paper_2410_01136_gb300.surrogate import Surrogate

    prob = inputs.config5_problem()
    sur = Surrogate.for_workload(batch=512, total_steps=steps, lr=1e-3, lr_min=1e-5)
    thetas = inputs.config5_thetas(n_maps, seed=50)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sur.dataset(prob, thetas)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = sur.train(steps, seed=1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    mean, scale = sur.normalization()

    hold = inputs.config5_thetas(512, seed=51)
    c = sur(torch.tensor(hold, dtype=torch.float32, device=dev))
    _, rms, fell = sur.judge(prob, hold, c, 1.0)
    base = torch.tensor(np.broadcast_to(mean.reshape(3, -1), (512, 3, sur.n_basis)).copy(), device=dev)
    _, rms0, _ = sur.judge(prob, hold, base, 1.0)
    rms, rms0 = rms.cpu().numpy(), rms0.cpu().numpy()

    # throughput: coefficients + d chi^2/d theta (VJP) for 16384 parameter sets per call
    B = 16384
    th = torch.tensor(inputs.config5_thetas(B, seed=52), dtype=torch.float32, device=dev)
    g = torch.randn((B, 3, sur.n_basis), device=dev)
    torch.cuda.nvtx.range_push("surrogate_eval")     # the warm-up calls: a profiler's filter for one call
    for _ in range(3):
        sur(th, g)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    n_rep = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n_rep):
        sur(th, g)
    e1.record()
    torch.cuda.synchronize()
    ms_call = e0.elapsed_time(e1) / n_rep
    sur.status()
    # dense FLOPs per parameter set: forward 2 sum(in*out) over the layers
    # (padded 64-wide input) and the input-gradient backward pass, the same
    # products without the first layer's weight gradient
    widths = (64,) + (1024,) * 4 + (3 * sur.n_basis,)
    fwd = sum(2 * widths[i] * widths[i + 1] for i in range(5))
    flop = B * (2 * fwd - 2 * 64 * 1024 + 2 * 16 * 1024)
    tf = flop / (ms_call * 1e-3) / 1e12
    peak = float(peaks.get("bf16_tflops", 1900.0))

    # the plain march's map + gradient on the same 408 MHz workload
    tgt = sx.forward(prob.with_theta(hold[1]))
    ws = torch.empty(max(sx.adjoint_workspace_bytes(prob), 1), dtype=torch.uint8, device=dev)
    p0 = prob.with_theta(hold[0])
    for _ in range(3):
        sx.adjoint(p0, target=tgt, sigma=0.5, workspace=ws)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(10):
        sx.adjoint(p0, target=tgt, sigma=0.5, workspace=ws)
    e1.record()
    torch.cuda.synchronize()
    ms_march = e0.elapsed_time(e1) / 10
    pass_all = float(np.mean(rms.max(axis=1) <= 1.0))

    # ensemble gate: a second network from other initial weights; draws where
    # the two disagree by more than 1 K (in-subspace RMS) go to the march
    sur_b = Surrogate.for_workload(batch=512, total_steps=steps, lr=1e-3, lr_min=1e-5, init_seed=8)
    sur_b.dataset(prob, thetas)
    sur_b.train(steps, seed=2)
    c_gate, dis = sur.gate(sur_b, torch.tensor(hold, dtype=torch.float32, device=dev))
    _, rms_g, _ = sur.judge(prob, hold, c_gate, 1.0)
    dis, rms_g = dis.cpu().numpy().max(axis=1), rms_g.cpu().numpy().max(axis=1)
    # calibrate the threshold on the first half of the held-out draws (largest
    # candidate with <= 1 % judged failures among accepted), report on the second
    cal, tst = slice(0, 256), slice(256, 512)
    tau = 0.0
    for cand in (0.05, 0.1, 0.15, 0.2, 0.25, 0.3, 0.4, 0.5, 0.75, 1.0):
        acc = dis[cal] <= cand
        if acc.any() and np.mean(rms_g[cal][acc] > 1.0) <= 0.01:
            tau = cand
    accepted = dis[tst] <= tau
    acc_frac = float(np.mean(accepted))
    fail_acc = float(np.mean(rms_g[tst][accepted] > 1.0)) if accepted.any() else None
    # gated cost per set: two surrogate evaluations + gradients, and the march
    # for the rejected share
    t_set = 2.0 * ms_call / B
    t_gated = t_set + (1.0 - acc_frac) * ms_march
    sur_b.close()
    out = {
        "workload": f"MLP 16->1024x4 (GELU)->3x3072, Nside 64 maps at 408 MHz, {n_maps} training maps, "
                    "+-20% parameter box, 512 held-out draws judged by the march",
        "dataset_s": t_data, "train_steps": steps, "train_s": t_train, "ms_per_train_step": 1e3 * t_train / steps,
        "final_loss": float(np.mean(losses[-200:])), "norm_scale_K": scale,
        "judged_rms_K": {s: {"median": float(np.median(rms[:, k])), "p90": float(np.percentile(rms[:, k], 90)),
                             "max": float(rms[:, k].max())} for k, s in enumerate("IQU")},
        "mean_map_rms_K": {s: {"median": float(np.median(rms0[:, k])), "p90": float(np.percentile(rms0[:, k], 90))}
                           for k, s in enumerate("IQU")},
        "pass_frac_1K_all_stokes": pass_all, "pass_frac_1K_I": float(np.mean(rms[:, 0] <= 1.0)),
        "fell_back_frac": float(fell.float().mean().item()),
        "gate": {"threshold_K": tau, "calibration": "largest threshold with <= 1 % judged failures among "
                 "accepted draws on held-out draws 0-255; figures below on draws 256-511",
                 "accepted_frac": acc_frac, "judged_fail_frac_among_accepted": fail_acc,
                 "judged_fail_frac_all_mean_prediction": float(np.mean(rms_g[tst] > 1.0)),
                 "maps_grad_per_s_gated": 1e3 / t_gated,
                 "speedup_vs_march_gated": ms_march / t_gated},
        "maps_grad_per_s": B / (ms_call * 1e-3), "batch": B, "ms_per_call": ms_call,
        "march_maps_grad_per_s_same_workload": 1e3 / ms_march,
        "speedup_vs_march": (B / (ms_call * 1e-3)) / (1e3 / ms_march),
        "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                     "flop_per_set": flop / B, "peak_basis": "bf16_tflops (burst) of the measured peaks file",
                     "kernels": "k_gemm_bf16 x 10, gather, seed scaling"},
        "l2": "activations of a 16384-set call ~1 GB > 129 MB L2",
    }
    sur.close()
    return out


def run_synax(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import paper_2410_01136_gb300 as sx
    from paper_2410_01136_gb300 import _native, inputs, tune
    sx.build()
    if args.only_hmc:
        if rank == 0:
            print(json.dumps({"hmc": bench_hmc(sx, inputs, torch, dev)}), flush=True)
        return
    if args.only_batch_low_res:
        tune.load_or_tune()
        chains = [p.replace(nside=16, n_steps=256) for p in inputs.config4()]
        if rank == 0:
            print(json.dumps({"batch_low_res": bench_batch(sx, inputs, torch, dev, n_runs=3, sets=chains,
                                                           name="256 chains, Nside 16, 256 steps")}), flush=True)
        return
    if args.only_wmap_stack:
        if rank == 0:
            print(json.dumps({"wmap_stack": bench_wmap_stack(sx, inputs, torch, dev, max(args.wmap_stack_runs, 1))}),
                  flush=True)
        return
    if args.only_grid:
        if rank == 0:
            print(json.dumps({"grid": bench_grid(sx, inputs, torch, dev, max(args.grid_runs, 1),
                                                 max(args.grid_runs, 1))}), flush=True)
        return
    if args.only_surrogate:
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                peaks = json.load(fh)
        except (OSError, ValueError):
            pass
        if rank == 0:
            print(json.dumps({"surrogate": bench_surrogate(sx, inputs, torch, dev, args.surrogate_steps, peaks,
                                                           args.surrogate_maps),
                              "surrogate_sh": bench_surrogate_sh(sx, inputs, torch, dev, args.surrogate_steps,
                                                                 args.surrogate_maps)}), flush=True)
        return
    if args.lanes:
        tune.reset()
        _native.check(_native.lib().synax_set_lanes_per_ray(-1, args.lanes), "synax_set_lanes_per_ray")
        lanes_table = {n: args.lanes for n in tune.STEP_BINS}
    else:
        lanes_table = tune.load_or_tune()      # launch width per step-count bin (cached per device)

    prob, th_target, sigma = inputs.config3(seed=3 + rank)
    # target: forward map of the perturbed parameters plus N(0, sigma^2) noise
    with torch.cuda.device(dev):
        target_clean = sx.forward(prob.with_theta(th_target))
        noise = torch.tensor(inputs.target_noise(tuple(target_clean.shape), seed=3 + rank, sigma=sigma),
                             dtype=torch.float32, device=dev)
        target = (target_clean + noise).contiguous()
    shape = tuple(target.shape)
    maps = torch.empty(shape, dtype=torch.float32, device=dev)
    ws = torch.empty(max(sx.adjoint_workspace_bytes(prob), 1), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def step():
        return sx.adjoint(prob, target=target, sigma=sigma, maps_out=maps, workspace=ws)

    def fwd():
        return sx.forward(prob, out=maps)

    for _ in range(max(args.warmup, 3)):
        step()
        fwd()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- timed region: K map+grad steps, L2 flushed between steps ----
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    peaks = measure_peaks(sx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # forward-only march of the same maps (context figure, same flushing)
    fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        fev[k][0].record(stream)
        fwd()
        fev[k][1].record(stream)
    torch.cuda.synchronize()
    fwd_ms = [a.elapsed_time(b) for a, b in fev]
    time.sleep(0.2)
    clk = clocks.stop()

    # ---- end to end through the public API with host buffers ----
    # Every step copies its target from pinned host memory, runs synax_adjoint
    # and copies maps, gradient and chi^2 back; two streams with their own
    # buffers alternate, so one step's copies overlap the other's kernels.
    # Each step also writes its own 256 MiB L2 flush, inside the timed region.
    h_target = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    h_target.copy_(target.cpu())
    streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    bufs = []
    for _ in range(2):
        bufs.append({"d_target": torch.empty(shape, dtype=torch.float32, device=dev),
                     "maps": torch.empty(shape, dtype=torch.float32, device=dev),
                     "ws": torch.empty(max(sx.adjoint_workspace_bytes(prob), 1), dtype=torch.uint8, device=dev),
                     "flush": torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev),
                     "h_maps": torch.empty(shape, dtype=torch.float32, pin_memory=True),
                     "h_grad": torch.empty(16, dtype=torch.float64, pin_memory=True),
                     "h_chi2": torch.empty(1, dtype=torch.float64, pin_memory=True)})

    def e2e_step(k):
        st, b = streams[k % 2], bufs[k % 2]
        with torch.cuda.stream(st):
            b["flush"].fill_(float(k))
            b["d_target"].copy_(h_target, non_blocking=True)
            g, c2 = sx.adjoint(prob, target=b["d_target"], sigma=sigma, maps_out=b["maps"], workspace=b["ws"])
            b["h_maps"].copy_(b["maps"], non_blocking=True)
            b["h_grad"].copy_(g, non_blocking=True)
            b["h_chi2"].copy_(c2, non_blocking=True)

    for k in range(4):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for st in streams:
        st.wait_event(e_start)
    for k in range(args.steps):
        e2e_step(k)
    for st in streams:
        ev = torch.cuda.Event()
        ev.record(st)
        stream.wait_event(ev)
    e_end.record(stream)
    barrier()
    e2e_ms = [e_start.elapsed_time(e_end) / args.steps]

    # the same call as a per-call latency: one stream, each step's copies,
    # kernels and read-back in sequence (no overlap between steps)
    b = bufs[0]
    lat = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        b["flush"].fill_(float(k))
        lat[k][0].record(stream)
        b["d_target"].copy_(h_target, non_blocking=True)
        g1, c1 = sx.adjoint(prob, target=b["d_target"], sigma=sigma, maps_out=b["maps"], workspace=b["ws"])
        b["h_maps"].copy_(b["maps"], non_blocking=True)
        b["h_grad"].copy_(g1, non_blocking=True)
        b["h_chi2"].copy_(c1, non_blocking=True)
        lat[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_lat_ms = float(np.median([a.elapsed_time(z) for a, z in lat]))

    ms = float(np.mean(step_ms))
    ms_e2e = float(np.mean(e2e_ms))
    ms_fwd = float(np.mean(fwd_ms))
    ms, ms_e2e, ms_fwd = slowest_rank_times([ms, ms_e2e, ms_fwd], device=dev)
    samples = prob.samples
    value = whole_job_rate(world, samples, ms)

    # roofline of the dominant kernel (the adjoint march): algorithmic FP32 and
    # MUFU work per launch over the launch's measured duration, against the
    # pipe peaks measured on this GPU inside the same clock-sampled region
    adj_fp32 = ADJ_FACTOR * FWD_FP32_OPS * samples
    adj_mufu = ADJ_FACTOR * FWD_MUFU_OPS * samples
    roof = roofline_alu(adj_fp32, adj_mufu, ms * 1e-3, peaks, "k_adjoint (+ k_reduce_partials)",
                        ADJ_FACTOR * FWD_EX2_OPS * samples)
    roof["traffic"] = ADJ_DRAM_BYTES
    roof["ops_per_sample"] = {"fp32": ADJ_FACTOR * FWD_FP32_OPS, "mufu": ADJ_FACTOR * FWD_MUFU_OPS,
                              "mufu_ex2": ADJ_FACTOR * FWD_EX2_OPS}
    fwd_roof = roofline_alu(FWD_FP32_OPS * samples, FWD_MUFU_OPS * samples, ms_fwd * 1e-3, peaks, "k_forward",
                            FWD_EX2_OPS * samples)

    out = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nside": 64, "n_steps": 512, "n_freq": 4, "n_theta": 16,
                   "samples_per_step": samples, "global_batch": world, "l2": "flushed between steps "
                   "(256 MiB write), inputs 2.4 MB", "parallelism": f"replicas x{world}"},
        "maps_grad_per_s": whole_job_rate(world, 1, ms),
        "forward_samples_per_s": whole_job_rate(world, samples, ms_fwd),
        "forward_ms": ms_fwd,
        "roofline": roof,
        "forward_roofline": fwd_roof,
        "peaks_measured": dict(peaks, sm_mhz=clk["sm_mhz"]),
        "clocks": clk,
        "e2e": {"value": whole_job_rate(world, samples, ms_e2e), "unit": "samples/s",
                "h2d_bytes_per_step": int(target.numel() * 4),
                "d2h_bytes_per_step": int(maps.numel() * 4 + 16 * 8 + 8),
                "ms_per_step": ms_e2e,
                "schedule": "two streams alternating steps (copies of one step overlap the other's kernels); "
                            "a 256 MiB L2 flush per step inside the timed region",
                "latency_ms_single_stream": e2e_lat_ms,
                "latency_note": "median per-call time on one stream: H2D target, synax_adjoint, D2H maps, "
                                "gradient and chi^2, no overlap between calls"},
        "gpu_launches": 2 * args.steps,
        "lanes_per_ray": {str(k): v for k, v in lanes_table.items()},
    }
    # the further rows are one-GPU measurements: reported from single-process runs only
    extras = rank == 0 and world == 1
    if extras and not args.no_batch:
        out["batch"] = bench_batch(sx, inputs, torch, dev)
        chains = [p.replace(nside=16, n_steps=256) for p in inputs.config4()]
        out["batch_low_res"] = bench_batch(sx, inputs, torch, dev, n_runs=20, sets=chains,
                                           name="256 chains, Nside 16, 256 steps, chi^2 map+gradient")
        out["gpu_launches_batch_per_run"] = 2
    if extras and not args.no_grid:
        out["grid"] = bench_grid(sx, inputs, torch, dev)
        out["interp_study"] = interp_study(sx, inputs, torch)
        out["wmap_stack"] = bench_wmap_stack(sx, inputs, torch, dev, max(args.wmap_stack_runs, 1))
        out["hmc"] = bench_hmc(sx, inputs, torch, dev)
    # every row against its kernel's roofline (same clock as the main line)
    for key in ("batch", "batch_low_res"):
        if key in out:
            out[key]["roofline"] = march_roofline("jf12", 4, out[key]["samples_per_s"], peaks, True,
                                                  "k_batch (+ k_batch_reduce)")
    if "grid" in out:
        g = out["grid"]
        g["roofline"] = march_roofline("grid", 1, g["samples_per_s"], peaks, True,
                                       "k_adjoint<GRID> (+ k_reduce_partials, k_grid_unpad)")
        g["forward_roofline"] = march_roofline("grid", 1, g["forward_samples_per_s"], peaks, False,
                                               "k_forward<GRID>")
    if "wmap_stack" in out:
        w = out["wmap_stack"]
        w["roofline"] = march_roofline("wmap_stack", 1, w["samples_per_s"], peaks, True,
                                       "k_adjoint<WMAP_STACK> (+ k_reduce_partials)")
        w["forward_roofline"] = march_roofline("wmap_stack", 1, w["forward_samples_per_s"], peaks, False,
                                               "k_forward<WMAP_STACK>")
    if "hmc" in out:
        h = out["hmc"]
        h["roofline"] = march_roofline("wmap", 1, h["gradient_evals_per_s"] * h["samples_per_map"], peaks,
                                       True, "k_batch<WMAP> per leapfrog step (momenta, leapfrog and "
                                             "Metropolis kernels included in the time)")
    if extras and not args.no_surrogate:
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                peaks = json.load(fh)
        except (OSError, ValueError):
            pass
        out["surrogate"] = bench_surrogate(sx, inputs, torch, dev, args.surrogate_steps, peaks, args.surrogate_maps)
        out["surrogate_sh"] = bench_surrogate_sh(sx, inputs, torch, dev, args.surrogate_steps, args.surrogate_maps)
    if extras and not args.no_cpu_baseline:
        try:
            rate, dt, threads, desc = oracle_map_grad_rate(16384)   # ~10 s on 16 cores
            rate1, dt1, _, desc1 = oracle_map_grad_rate(1024, threads=1)   # ~10 s on one core
            out["cpu_baseline"] = {"value": rate, "unit": "samples/s", "cores": threads,
                                   "kind": "oracle", "sample": desc, "seconds": dt,
                                   "value_1thread": rate1, "sample_1thread": desc1, "seconds_1thread": dt1,
                                   "nproc": os.cpu_count(), "cpu_model": cpu_model()}
        except Exception as exc:  # the oracle is a baseline; report why it is absent
            out["cpu_baseline"] = {"value": None, "unit": "samples/s", "cores": os.cpu_count(),
                                   "kind": "oracle", "sample": f"failed: {exc}"}
        # the oracle beside each further row, on bounded samples (~1-3 s each)
        try:
            for key in ("batch", "batch_low_res"):
                if key in out:
                    out[key]["oracle"] = {"samples_per_s": out["cpu_baseline"]["value"],
                                          "note": "the sets are JF12-type maps at 4 frequencies: the "
                                                  "oracle's rate per LOS sample is cpu_baseline's"}
            if "grid" in out:
                out["grid"]["oracle"] = oracle_row(
                    inputs.grid_problem(), 8192, range(3),
                    "map + theta gradient; the oracle's central differences of the 1.57 M grid values "
                    "would take 3.1 M maps")
            if "wmap_stack" in out:
                out["wmap_stack"]["oracle"] = oracle_row(inputs.wmap_stack_problem(), 2048, range(19))
            if "hmc" in out:
                out["hmc"]["oracle"] = oracle_row(hmc_problem(inputs), 8192, range(4),
                                                  "one gradient evaluation = map + 8 difference maps")
        except Exception as exc:
            out["oracle_rows_error"] = str(exc)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_synax(args)


if __name__ == "__main__":
    main()
