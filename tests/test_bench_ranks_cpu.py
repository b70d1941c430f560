"""The benchmark's multi-rank bookkeeping on CPU ranks (gloo, world size 2):
every rank's per-step times are replaced by their maximum over the ranks,
the whole-job rate is all ranks' units over the slowest rank's time, and
the reference arm does its work on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r measured (1 + r, 5 - r, 2) ms for (step, end to end, forward)
        got = bench.slowest_rank_times([1.0 + rank, 5.0 - rank, 2.0], device="cpu")
        np.save(f"{out_path}.{rank}.npy", np.array(got))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slowest_rank_times_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "times")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        assert np.array_equal(np.load(f"{out}.{r}.npy"), [2.0, 5.0, 2.0])


def test_single_process_and_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_times([1.5, 2.5]) == [1.5, 2.5]
    # weak scaling: 4 ranks of 25 165 824 samples in 0.605 ms
    assert bench.whole_job_rate(4, 25165824, 0.605) == pytest.approx(4 * 25165824 / 0.605e-3, rel=1e-15)


def test_reference_arm_runs_on_rank_0_only():
    """Under torchrun a rank other than 0 prints nothing and exits 0 without
    running the oracle."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_gpu_arm_fails_loudly_without_a_gpu():
    """The product path has no CPU fallback: without CUDA the GPU arm exits
    non-zero instead of printing a number."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "1", "--warmup", "0",
                        "--no-batch", "--no-grid", "--no-surrogate", "--no-cpu-baseline"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    for line in r.stdout.splitlines():
        assert "value" not in json.loads(line) if line.startswith("{") else True


def test_roofline_accounting():
    """The per-sample operation counts behind every row's roofline and the
    choice of bounding pipe against given peaks: the JF12-type adjoint is
    3 x (200 FP32 + 22 MUFU, 9 of them ex2) at four frequencies; the grid
    adjoint adds 36 FP32 of node weights.  Each pipe's roofline time is its
    operations over its rates (ex2 and the other SFU instructions apart),
    the longer one bounds, frac = that time over the measured time."""
    sys.path.insert(0, ROOT)
    import bench
    peaks = {"fp32_top": 40.0, "mufu_ex2": 10.0, "mufu_other": 5.0}
    r = bench.march_roofline("jf12", 4, 4.0e10, peaks, True, "k")
    assert r["ops_per_sample"] == {"fp32": 600, "mufu": 66, "mufu_ex2": 27} and r["pipe"] == "FP32"
    assert r["peak"] == pytest.approx(40.0)
    assert r["frac"] == pytest.approx(4.0e10 * 600 / 40.0e12)
    assert r["frac_other_pipe"] == pytest.approx(4.0e10 * (27 / 10.0e12 + 39 / 5.0e12))
    f = bench.march_roofline("jf12", 4, 1.0e11, peaks, False, "k")
    assert f["ops_per_sample"] == {"fp32": 200, "mufu": 22, "mufu_ex2": 9}
    g = bench.march_roofline("grid", 1, 1.0, peaks, True, "k")
    assert g["ops_per_sample"] == {"fp32": 486, "mufu": 33, "mufu_ex2": 15} and g["pipe"] == "FP32"
    for model, fwd in (("wmap", {"fp32": 68, "mufu": 16, "mufu_ex2": 6}),
                       ("wmap_stack", {"fp32": 107, "mufu": 27, "mufu_ex2": 5})):
        w = bench.march_roofline(model, 1, 1.0e10, peaks, False, "k")
        assert w["ops_per_sample"] == fwd and w["pipe"] == "MUFU"
        t_mufu = fwd["mufu_ex2"] / 10.0e12 + (fwd["mufu"] - fwd["mufu_ex2"]) / 5.0e12
        assert w["frac"] == pytest.approx(1.0e10 * t_mufu)
        assert w["peak"] == pytest.approx(fwd["mufu"] / t_mufu / 1e12)
    # a faster SFU moves the stacked model's bound to the FP32 pipe
    w = bench.march_roofline("wmap_stack", 1, 1.0e10, {"fp32_top": 40.0, "mufu_ex2": 20.0, "mufu_other": 12.0},
                             False, "k")
    assert w["pipe"] == "FP32" and w["frac"] == pytest.approx(1.0e10 * 107 / 40.0e12)
