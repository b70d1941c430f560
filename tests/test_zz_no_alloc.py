"""synax_adjoint_noalloc: the adjoint for callers that cannot allocate device
memory (its scratch is a fixed array inside the library).  Checked through
the C ABI against synax_adjoint with a caller-provided workspace, on two
calls in a row (the second reuses the array the first one left behind).

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2410_01136_gb300 import _native, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_01136_gb300 import build
    build()
    oracle.build()
    return _t


def ptr(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def call_reference(torch, L, s, gm, tgt, sigma):
    n = ctypes.c_size_t(0)
    assert L.synax_adjoint_workspace_bytes(ctypes.byref(s), ctypes.byref(n)) == 0
    ws = torch.empty(max(n.value, 1), dtype=torch.uint8, device="cuda")
    g = torch.empty(s.n_theta, dtype=torch.float64, device="cuda")
    c = torch.empty(1, dtype=torch.float64, device="cuda")
    m = torch.empty_like(tgt if tgt is not None else gm)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.synax_adjoint(ctypes.byref(s), ptr(gm), ptr(tgt), sigma, ptr(g), ptr(c), ptr(m), ptr(ws),
                         ws.numel(), stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    return g.cpu().numpy(), c.cpu().numpy(), m.cpu().numpy()


def call_noalloc(torch, L, s, gm, tgt, sigma):
    g = torch.full((s.n_theta,), float("nan"), dtype=torch.float64, device="cuda")
    c = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    m = torch.full_like(tgt if tgt is not None else gm, float("nan"))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.synax_adjoint_noalloc(ctypes.byref(s), ptr(gm), ptr(tgt), sigma, ptr(g), ptr(c), ptr(m),
                                 stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    return g.cpu().numpy(), c.cpu().numpy(), m.cpu().numpy()


def close(a, b):
    # the gradient tolerance of the adjoint tests, relative to the reference
    return np.all(np.abs(a - b) <= 1e-3 * np.abs(b) + 1e-4 * np.max(np.abs(b)))


def test_noalloc_matches_workspace_adjoint(torch):
    L = _native.lib()
    prob, th_target, sigma = inputs.config3()
    prob = prob.replace(nside=16, n_steps=128)
    target = oracle.forward(prob.with_theta(th_target)) + inputs.target_noise((4, 3, prob.npix), seed=3)
    tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
    s = _native.problem_struct(prob)
    g_ref, c_ref, m_ref = call_reference(torch, L, s, None, tgt, sigma)
    for _ in range(2):                       # two calls in a row share the static scratch
        g, c, m = call_noalloc(torch, L, s, None, tgt, sigma)
        assert close(g, g_ref)
        assert c[0] == pytest.approx(c_ref[0], rel=1e-6)
        assert np.allclose(m, m_ref, rtol=1e-6, atol=1e-6 * np.abs(m_ref).max())
    # VJP mode, two calls in a row
    gm = torch.tensor(inputs.normal(5, 4 * 3 * prob.npix).reshape(4, 3, prob.npix),
                      dtype=torch.float32, device="cuda")
    gv_ref, _, _ = call_reference(torch, L, s, gm, None, 1.0)
    for _ in range(2):
        gv, _, _ = call_noalloc(torch, L, s, gm, None, 1.0)
        assert close(gv, gv_ref)


def max_pixels_within_limit(L, prob):
    """Largest pixel count whose adjoint workspace fits the library's fixed
    scratch (bisection on synax_adjoint_workspace_bytes, a host-only call)."""
    limit = 8 << 20
    lo, hi = 1, prob.npix
    while lo < hi:
        mid = (lo + hi + 1) // 2
        s = _native.problem_struct(prob.replace(pix_begin=0, pix_count=mid))
        n = ctypes.c_size_t(0)
        assert L.synax_adjoint_workspace_bytes(ctypes.byref(s), ctypes.byref(n)) == 0
        if n.value <= limit:
            lo = mid
        else:
            hi = mid - 1
    return lo


def test_noalloc_at_the_size_limit(torch):
    """The largest pixel range that fits, at 32 lanes per ray (the most CTAs,
    so the last CTA's partial row sits at the end of the array), against the
    workspace adjoint; one pixel more is rejected before anything runs."""
    L = _native.lib()
    base = inputs.config2().replace(nside=256, n_steps=16)
    n_max = max_pixels_within_limit(L, base)
    assert 200000 < n_max < base.npix
    prob = base.replace(pix_begin=base.npix - n_max - 5, pix_count=n_max)
    s = _native.problem_struct(prob)
    gm = torch.tensor(inputs.normal(6, 4 * 3 * n_max).reshape(4, 3, n_max), dtype=torch.float32, device="cuda")
    assert L.synax_set_lanes_per_ray(-1, 32) == 0
    try:
        g_ref, _, _ = call_reference(torch, L, s, gm, None, 1.0)
        for _ in range(2):
            g, _, _ = call_noalloc(torch, L, s, gm, None, 1.0)
            assert close(g, g_ref)
    finally:
        assert L.synax_set_lanes_per_ray(-1, 0) == 0
    over = _native.problem_struct(base.replace(pix_begin=0, pix_count=n_max + 1))
    g = torch.full((16,), 7.0, dtype=torch.float64, device="cuda")
    rc = L.synax_adjoint_noalloc(ctypes.byref(over), ptr(gm), None, 1.0, ptr(g), None, None,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _native.SYNAX_ESPACE
    assert torch.all(g == 7.0)                  # nothing was enqueued


def test_noalloc_fp64_wmap(torch):
    """The FP64 march and the 8-parameter WMAP-type model through the scratch."""
    L = _native.lib()
    prob = inputs.config1().replace(nside=8, n_steps=64)
    assert prob.f64
    target = oracle.forward(prob) + inputs.target_noise((prob.n_freq, 3, prob.npix), seed=12, sigma=0.1)
    tgt = torch.tensor(target, dtype=torch.float64, device="cuda")
    s = _native.problem_struct(prob)
    g_ref, c_ref, m_ref = call_reference(torch, L, s, None, tgt, 0.1)
    for _ in range(2):
        g, c, m = call_noalloc(torch, L, s, None, tgt, 0.1)
        assert np.allclose(g, g_ref, rtol=1e-12, atol=1e-12 * np.abs(g_ref).max())
        assert c[0] == pytest.approx(c_ref[0], rel=1e-12)
        assert np.allclose(m, m_ref, rtol=1e-12, atol=0)


def test_noalloc_rejects_oversize(torch):
    L = _native.lib()
    big = _native.problem_struct(inputs.config2().replace(nside=256, n_steps=16))
    g = torch.empty(16, dtype=torch.float64, device="cuda")
    dummy = torch.empty(1, dtype=torch.float32, device="cuda")
    rc = L.synax_adjoint_noalloc(ctypes.byref(big), ptr(dummy), None, 1.0, ptr(g), None, None,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _native.SYNAX_ESPACE
