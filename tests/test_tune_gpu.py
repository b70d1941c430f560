"""Autotuner of the launch width and its effect: every width gives the same
maps up to FP32 rounding, and the tuned table is installed and cached."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2410_01136_gb300 import adjoint, forward, inputs, tune

from .parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_01136_gb300 import build
    build()
    oracle.build()
    yield _t
    tune.reset()


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_every_width_matches_the_oracle(torch, lanes):
    from paper_2410_01136_gb300 import set_lanes_per_ray
    prob = inputs.config2().replace(nside=8, n_steps=200)
    set_lanes_per_ray(lanes)
    try:
        g = forward(prob).cpu().numpy()
        tg = torch.zeros((4, 3, prob.npix), device="cuda")
        grad, _ = adjoint(prob, target=tg, sigma=0.5)
    finally:
        set_lanes_per_ray(0)
    assert_parity(g, oracle.forward(prob), what=f"{lanes} lanes per ray")
    ref, _ = adjoint(prob, target=tg, sigma=0.5)
    ref = ref.cpu().numpy()
    assert np.allclose(grad.cpu().numpy(), ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def test_tune_installs_and_caches(torch, tmp_path):
    path = str(tmp_path / "tune.json")
    table = tune.load_or_tune(path)
    assert set(table) == set(tune.STEP_BINS)
    assert all(v in tune.CANDIDATES for v in table.values())
    with open(path) as fh:
        cache = json.load(fh)
    assert torch.cuda.get_device_name() in cache
    again = tune.load_or_tune(path)           # from the cache, no timing
    assert again == table
