"""Autotuner of the launch width: how many lanes of a warp march one ray.

For each step-count bin of the library's tuning table (edges 64, 128, 256,
512, 1024, 2048, 4096) it times the map+gradient march (synax_adjoint, chi^2
mode) of a representative map at 8, 16 and 32 lanes per ray with CUDA
events, installs the fastest through synax_set_lanes_per_ray and caches the
table per device name in a JSON file ($SYNAX_TUNE_CACHE, default
~/.cache/synax_lanes_per_ray.json).  Results do not depend on the width
beyond FP32 rounding; only speed does.
"""
from __future__ import annotations

import json
import os

from . import _native, inputs
from ._native import check, lib

CANDIDATES = (8, 16, 32)
STEP_BINS = (64, 128, 256, 512, 1024, 2048)


def cache_path() -> str:
    return os.environ.get("SYNAX_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "synax_lanes_per_ray.json"))


def install(table: dict) -> None:
    """Install {n_steps_bin: lanes} into the library's tuning table."""
    for n_steps, lanes in table.items():
        check(lib().synax_set_lanes_per_ray(int(n_steps), int(lanes)), "synax_set_lanes_per_ray")


def reset() -> None:
    check(lib().synax_set_lanes_per_ray(-1, 0), "synax_set_lanes_per_ray")
    for n in STEP_BINS:
        check(lib().synax_set_lanes_per_ray(n, 0), "synax_set_lanes_per_ray")


def measure(nside: int = 64, step_bins=STEP_BINS, repeats: int = 5) -> dict:
    """Milliseconds per map+gradient for every (bin, width): {n: {lanes: ms}}."""
    import torch

    import paper_2410_01136_gb300 as sx
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream(dev)
    out = {}
    for n_steps in step_bins:
        prob, _, sigma = inputs.config3()
        prob = prob.replace(nside=nside, n_steps=n_steps)
        target = torch.zeros((prob.n_freq, 3, prob.npix), dtype=torch.float32, device="cuda")
        ws = torch.empty(max(sx.adjoint_workspace_bytes(prob), 1), dtype=torch.uint8, device="cuda")
        res = {}
        for lanes in CANDIDATES:
            check(lib().synax_set_lanes_per_ray(-1, lanes), "synax_set_lanes_per_ray")
            for _ in range(2):
                sx.adjoint(prob, target=target, sigma=sigma, workspace=ws)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(repeats):
                sx.adjoint(prob, target=target, sigma=sigma, workspace=ws)
            e1.record(stream)
            torch.cuda.synchronize()
            res[lanes] = e0.elapsed_time(e1) / repeats
        out[n_steps] = res
    check(lib().synax_set_lanes_per_ray(-1, 0), "synax_set_lanes_per_ray")
    return out


def tune(nside: int = 64, step_bins=STEP_BINS, repeats: int = 5) -> dict:
    """Measure, install and return {n_steps_bin: best lanes}."""
    times = measure(nside, step_bins, repeats)
    table = {n: min(r, key=r.get) for n, r in times.items()}
    install(table)
    return table


def load_or_tune(path: str | None = None, retune: bool = False) -> dict:
    """Install the cached table for this device, tuning (and caching) it first
    if there is none."""
    import torch
    path = path or cache_path()
    name = torch.cuda.get_device_name()
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
    if not retune and name in cache:
        table = {int(k): int(v) for k, v in cache[name].items()}
        install(table)
        return table
    table = tune()
    cache[name] = {str(k): v for k, v in table.items()}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as fh:
            json.dump(cache, fh, indent=1)
    except OSError:
        pass
    return table
