"""Spreading the march over several GPUs (one process per GPU).

The path partitions two ways:
  * independent parameter sets (maps, HMC chains): each rank marches its own
    sets (`set_range`) -- weak scaling, no collective at all;
  * one large map: each rank marches a contiguous range of RING pixels
    (`pixel_range`, the ABI's pix_begin / pix_count).  chi^2 (Eq. 15 up to
    its constant) and its gradient are sums over pixels, so the ranks' partial
    results combine by one all-reduce of n_theta + 1 doubles
    (`allreduce_grad`), the only exchange.
"""
from __future__ import annotations


def pixel_range(npix: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced [begin, begin + count) of rank `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or npix < 0:
        raise ValueError("bad world / rank / npix")
    base, extra = divmod(npix, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def set_range(n_sets: int, world: int, rank: int) -> range:
    """The parameter sets of rank `rank` under the same balanced split."""
    begin, count = pixel_range(n_sets, world, rank)
    return range(begin, begin + count)


def shard_problem(prob, world: int, rank: int):
    """The problem restricted to this rank's pixel range."""
    begin, count = pixel_range(prob.npix, world, rank)
    return prob.replace(pix_begin=begin, pix_count=count)


def shard_maps(maps, prob, world: int, rank: int):
    """This rank's slice [F][3][count] of full-sky maps [F][3][npix]."""
    begin, count = pixel_range(prob.npix, world, rank)
    return maps[..., begin:begin + count]


def allreduce_grad(grad, chi2, group=None):
    """Sum the ranks' (gradient, chi^2) in one all-reduce; returns the totals.
    grad: tensor [n_theta] (float64); chi2: tensor [1] or scalar tensor."""
    import torch
    import torch.distributed as dist
    buf = torch.cat([grad.reshape(-1).to(torch.float64), chi2.reshape(-1).to(torch.float64)])
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf[:-1].to(grad.dtype), buf[-1:].reshape(chi2.shape).to(chi2.dtype)


def sharded_chi2_grad(prob, target, sigma: float, world: int, rank: int, group=None):
    """chi^2 map + gradient of the full map, this rank marching its pixel range
    on its own GPU (synax_adjoint), combined over the ranks."""
    import torch

    from . import adjoint
    sub = shard_problem(prob, world, rank)
    tgt = shard_maps(target, prob, world, rank).contiguous()
    g, c2 = adjoint(sub, target=tgt, sigma=sigma)
    return allreduce_grad(g, c2, group)

