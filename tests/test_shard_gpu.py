"""Pixel-range shards of one map, marched one after another on one GPU: their
(gradient, chi^2) sum to the full-map adjoint (what the all-reduce of a
multi-GPU run combines)."""
import numpy as np
import pytest

from paper_2410_01136_gb300 import inputs, shard

pytestmark = pytest.mark.gpu


def test_shards_sum_to_full_map():
    import torch
    import paper_2410_01136_gb300 as sx
    sx.build()
    prob = inputs.config2().replace(nside=8, n_steps=128)
    target = sx.forward(prob.with_theta(inputs.perturbed_theta(prob.theta, seed=3))).contiguous()
    g_full, c_full = sx.adjoint(prob, target=target, sigma=0.5)
    world = 3
    g_sum = torch.zeros_like(g_full)
    c_sum = torch.zeros_like(c_full)
    for r in range(world):
        g, c = shard.sharded_chi2_grad(prob, target, 0.5, world, r)
        g_sum += g
        c_sum += c
    g_full, g_sum = g_full.cpu().numpy(), g_sum.cpu().numpy()
    assert abs(float(c_sum.item()) - float(c_full.item())) <= 1e-6 * abs(float(c_full.item()))
    assert np.allclose(g_sum, g_full, rtol=1e-5, atol=1e-6 * np.max(np.abs(g_full)))
