"""Multi-rank decomposition on CPU ranks (gloo, world size 2): pixel ranges
partition the map, and the all-reduce of per-shard (gradient, chi^2) equals
the full-map result.  The per-shard values come from the FP64 oracle, standing
in for each rank's GPU march."""
import os
import socket

import numpy as np
import pytest

from paper_2410_01136_gb300 import inputs, shard


@pytest.mark.parametrize("npix,world", [(48, 2), (49, 2), (3072, 3), (5, 8), (0, 2)])
def test_pixel_ranges_partition(npix, world):
    seen = []
    sizes = []
    for r in range(world):
        b, c = shard.pixel_range(npix, world, r)
        seen.extend(range(b, b + c))
        sizes.append(c)
    assert seen == list(range(npix))
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.pixel_range(npix, world, world)


def _problem():
    return inputs.config2().replace(nside=2, n_steps=32, freq_hz=(1.4e9,))


def _chi2_grad(prob, target, pix):
    import oracle
    theta = np.asarray(prob.theta, dtype=np.float64)
    scale = inputs.jf12_scales(theta)

    def chi2(th):
        m = oracle.forward(prob.with_theta(th), pix=pix, threads=1)
        return oracle.chi2(m, target[..., pix], 0.5)

    g = oracle.fd_gradient(chi2, theta, 1e-4 * scale)
    return g, chi2(theta)


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _problem()
        import oracle
        target = oracle.forward(prob.with_theta(inputs.perturbed_theta(prob.theta, seed=3)), threads=1)
        b, c = shard.pixel_range(prob.npix, world, rank)
        g, c2 = _chi2_grad(prob, target, np.arange(b, b + c))
        tg, tc = shard.allreduce_grad(torch.tensor(g, dtype=torch.float64), torch.tensor([c2], dtype=torch.float64))
        if rank == 0:
            np.save(out_path, np.concatenate([tg.numpy(), tc.numpy()]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_chi2_gradient_equals_full_map(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    oracle.build()
    out = str(tmp_path / "reduced.npy")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    prob = _problem()
    target = oracle.forward(prob.with_theta(inputs.perturbed_theta(prob.theta, seed=3)), threads=1)
    g, c2 = _chi2_grad(prob, target, np.arange(prob.npix))
    assert abs(got[-1] - c2) <= 1e-12 * abs(c2)
    assert np.allclose(got[:-1], g, rtol=1e-9, atol=1e-12 * np.max(np.abs(g)))


def test_shard_problem_and_maps():
    prob = inputs.config2().replace(nside=4)
    maps = np.arange(2 * 3 * prob.npix).reshape(2, 3, prob.npix)
    parts = [shard.shard_maps(maps, prob, 3, r) for r in range(3)]
    assert np.array_equal(np.concatenate(parts, axis=-1), maps)
    sub = shard.shard_problem(prob, 3, 1)
    assert (sub.pix_begin, sub.pix_count) == shard.pixel_range(prob.npix, 3, 1)
