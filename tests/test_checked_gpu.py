"""SYNAX_CHECKED and the device status word (synax_last_status) on the GPU.

Every case here is in bounds: a checked launch must give results identical
to the unchecked launch (the checks only test indexes) and leave the status
word clear.  The one recorded error comes from the bounded-wait self-test,
whose wait runs out by design: synax_last_status returns SYNAX_ETIMEOUT
with the GEMM-wait site once, and SYNAX_OK on the next read (the read
clears the word).  No test makes an index go out of bounds on the device:
the host validation forbids it, and the predicate itself is checked on the
host (tests/test_abi_cpu.py)."""
import ctypes

import numpy as np
import pytest

from paper_2410_01136_gb300 import (BatchPlan, _native, adjoint, adjoint_grid, forward, inputs,
                                    last_status)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_01136_gb300 import build
    build()
    last_status()                      # start from a clear word
    return _t


@pytest.mark.parametrize("prob", [
    inputs.config2().replace(nside=8, n_steps=100, pix_begin=17, pix_count=601),
    inputs.config1().replace(nside=4, n_steps=40),
    inputs.grid_problem(nside=4, n_steps=48, freq_hz=(408e6, 2.4e9), n=(9, 7, 4)),
    inputs.wmap_stack_problem(nside=4, n_steps=33, freq_hz=(1.4e9,)),
], ids=["jf12", "wmap_f64", "grid", "wmap_stack"])
def test_checked_forward_identical(torch, prob):
    a = forward(prob).cpu().numpy()
    b = forward(prob.replace(checked=True)).cpu().numpy()
    assert last_status() == (0, 0, 0)
    assert np.array_equal(a, b)


def test_checked_adjoint_identical(torch):
    prob = inputs.config2().replace(nside=8, n_steps=64)
    tgt = forward(prob.with_theta(inputs.perturbed_theta(prob.theta, seed=5)))
    g0, c0 = adjoint(prob, target=tgt, sigma=0.5)
    m1 = torch.empty_like(tgt)
    g1, c1 = adjoint(prob.replace(checked=True), target=tgt, sigma=0.5, maps_out=m1)
    assert last_status() == (0, 0, 0)
    assert torch.equal(g0, g1) and torch.equal(c0, c1)
    assert torch.equal(m1, forward(prob))


def test_checked_grid_adjoint(torch):
    prob = inputs.grid_problem(nside=4, n_steps=48, freq_hz=(2.4e9,), n=(9, 7, 4))
    gm = torch.tensor(inputs.normal(inputs.substream(3, 1), 3 * prob.npix).reshape(1, 3, prob.npix),
                      dtype=torch.float32, device="cuda")
    g0, gg0 = adjoint_grid(prob, gmaps=gm)
    g1, gg1 = adjoint_grid(prob.replace(checked=True), gmaps=gm)
    assert last_status() == (0, 0, 0)
    assert torch.equal(g0, g1)
    # the grid gradient is summed with atomic adds (order not fixed)
    assert torch.allclose(gg0, gg1, rtol=1e-5, atol=1e-6 * gg0.abs().max().item())


def test_checked_batch_identical(torch):
    sets = [s.replace(nside=(2, 4)[i % 2], n_steps=(32, 77)[i % 2]) for i, s in enumerate(inputs.config4(n_sets=4))]
    tg = [forward(s.with_theta(inputs.perturbed_theta(s.theta, seed=9 + i))) for i, s in enumerate(sets)]
    p0 = BatchPlan(sets)
    g0, c0 = p0.run(targets=tg, sigma=0.5)
    p1 = BatchPlan([s.replace(checked=True) for s in sets])
    g1, c1 = p1.run(targets=tg, sigma=0.5)
    assert last_status() == (0, 0, 0)
    assert torch.equal(g0, g1) and torch.equal(c0, c1)
    p0.close()
    p1.close()


def test_timeout_reaches_the_status_word(torch):
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    cycles = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = _native.lib().synax_wait_selftest(ctypes.c_void_p(err.data_ptr()), ctypes.c_void_p(cycles.data_ptr()),
                                           ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0
    code, site, _ = last_status(stream)
    assert code == _native.SYNAX_ETIMEOUT and site == _native.SITE_GEMM_WAIT
    assert int(err.item()) == 1
    assert last_status(stream) == (0, 0, 0)             # the read cleared it
