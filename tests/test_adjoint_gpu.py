"""Gradients of the CUDA adjoint march (synax_adjoint through the C ABI)
against central finite differences of the FP64 oracle.

Reference: central differences with h_i = 1e-4 s_i (s_i = |theta_i|, 3 uG for
arm strengths), Richardson-extrapolated from h and h/2.  At 408 MHz the
Faraday phase reaches ~10^3 rad, so a plain central difference at 1e-4
relative carries up to ~1e-3 relative truncation error; the extrapolation
removes its h^2 term.  Tolerance per component:
|g - g_FD| <= 1e-3 |g_FD| + 1e-4 max_j |g_FD,j| (FP32 march); FP64 marches
are held to 1e-6 / 1e-7.
"""
import numpy as np
import pytest

import oracle
from paper_2410_01136_gb300 import SynaxMaps, adjoint, forward, inputs

from .parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_01136_gb300 import build
    build()
    oracle.build()
    return _t


def scales(prob):
    if prob.model_id == inputs.MODEL_JF12:
        return inputs.jf12_scales(prob.theta)
    s = np.abs(prob.theta).copy()
    s[s == 0] = 1.0          # WMAP psi1, chi0B at zero: absolute steps
    return s


def fd_reference(prob, loss, pix=None):
    """Richardson-extrapolated central differences of loss(oracle maps)."""
    th = prob.theta
    h = 1e-4 * scales(prob)

    def L(t):
        return loss(oracle.forward(prob.with_theta(t), pix=pix))

    g1 = oracle.fd_gradient(L, th, h)
    g2 = oracle.fd_gradient(L, th, h / 2)
    return (4 * g2 - g1) / 3, g1


def assert_grad(g, ref, rel=1e-3, floor=1e-4, what=""):
    g = np.asarray(g, dtype=np.float64)
    tol = rel * np.abs(ref) + floor * np.max(np.abs(ref))
    bad = np.where(np.abs(g - ref) > tol)[0]
    assert bad.size == 0, (what, [(int(i), float(g[i]), float(ref[i])) for i in bad])


def seeds(prob, seed=7, pix=None):
    n = prob.n_pix_out
    g = inputs.normal(inputs.substream(seed, n), prob.n_freq * 3 * n).reshape(prob.n_freq, 3, n)
    # scale each frequency's seeds to the map's magnitude so all terms matter
    if pix is not None:
        mask = np.zeros(n, dtype=bool)
        mask[pix] = True
        g[:, :, ~mask] = 0.0
    return g


@pytest.mark.parametrize("f64", [False, True])
def test_vjp_jf12_small(torch, f64):
    prob = inputs.config2().replace(nside=4, n_steps=64, f64=f64)
    gm = seeds(prob)
    dt = torch.float64 if f64 else torch.float32
    g = adjoint(prob, gmaps=torch.tensor(gm, dtype=dt, device="cuda")).cpu().numpy()
    ref, _ = fd_reference(prob, lambda m: float(np.sum(gm * m)))
    if f64:
        assert_grad(g, ref, 1e-6, 1e-7, "JF12 VJP FP64")
    else:
        assert_grad(g, ref, what="JF12 VJP FP32")


@pytest.mark.parametrize("f64", [False, True])
def test_vjp_wmap_small(torch, f64):
    prob = inputs.config1().replace(nside=4, n_steps=64, f64=f64)
    th = prob.theta.copy()
    th[2], th[3] = 0.05, 0.3            # exercise the psi1 and chi0B derivatives
    prob = prob.with_theta(th)
    gm = seeds(prob, seed=8)
    dt = torch.float64 if f64 else torch.float32
    g = adjoint(prob, gmaps=torch.tensor(gm, dtype=dt, device="cuda")).cpu().numpy()
    ref, _ = fd_reference(prob, lambda m: float(np.sum(gm * m)))
    if f64:
        assert_grad(g, ref, 1e-6, 1e-7, "WMAP VJP FP64")
    else:
        assert_grad(g, ref, what="WMAP VJP FP32")


def chi2_problem(nside, n_steps):
    prob, th_target, sigma = inputs.config3()
    prob = prob.replace(nside=nside, n_steps=n_steps)
    target = oracle.forward(prob.with_theta(th_target))
    target = target + inputs.target_noise(target.shape, seed=3, sigma=sigma)
    return prob, target, sigma


# 3 and 13 steps give lane chunks of 0-1 and 1-2 samples at 8 lanes per ray
# (a lone sample pairs with a masked placeholder in the two-sample reverse
# pass); 100 gives chunks of 12 and 13
@pytest.mark.parametrize("n_steps", [3, 13, 64, 100])
def test_chi2_jf12(torch, n_steps):
    prob, target, sigma = chi2_problem(8, n_steps)
    maps = torch.empty((4, 3, prob.npix), device="cuda")
    grad, chi2 = adjoint(prob, target=torch.tensor(target, dtype=torch.float32, device="cuda"),
                         sigma=sigma, maps_out=maps)
    g = grad.cpu().numpy()
    ora_maps = oracle.forward(prob)
    chi2_ora = oracle.chi2(ora_maps, target, sigma)
    assert float(chi2.item()) == pytest.approx(chi2_ora, rel=1e-5)
    ref, _ = fd_reference(prob, lambda m: oracle.chi2(m, target, sigma))
    assert_grad(g, ref, what=f"chi2 JF12 N={n_steps}")
    # maps_out is the map: against the oracle at the stated tolerance, and
    # against the forward kernel (the same arithmetic, compiled separately
    # under another register budget, so FMA contraction may differ: I agrees
    # to rounding; Q+iU, which cancels by up to ~100x at 408 MHz, to 1e-5)
    assert_parity(maps.cpu().numpy(), ora_maps, what="adjoint maps_out vs oracle")
    fwd = forward(prob).cpu().numpy()
    assert_parity(maps.cpu().numpy(), fwd, 1e-6, 1e-5, "adjoint maps_out vs forward")


def test_chi2_jf12_max_sizes(torch):
    """The chi^2 gradient at the ABI's largest Nside (8192: pixel runs at
    the polar-cap boundary and at the last pixel) and largest step count
    (65536), against Richardson differences of the oracle on those pixels."""
    npix = 12 * 8192 ** 2
    ncap = 2 * 8192 * (8192 - 1)
    cases = [(inputs.config2().replace(nside=8192, n_steps=64), ncap - 24, 48),
             (inputs.config2().replace(nside=8192, n_steps=64), npix - 32, 32),
             (inputs.config2().replace(nside=2, n_steps=65536), 20, 6)]
    for base, begin, count in cases:
        pix = np.arange(begin, begin + count)
        th_t = inputs.perturbed_theta(base.theta, seed=9)
        target = oracle.forward(base.with_theta(th_t), pix=pix)
        target = target + inputs.target_noise(target.shape, seed=10, sigma=0.5)
        prob = base.replace(pix_begin=begin, pix_count=count)
        grad, chi2 = adjoint(prob, target=torch.tensor(target, dtype=torch.float32, device="cuda"), sigma=0.5)
        maps = oracle.forward(base, pix=pix)
        assert float(chi2.item()) == pytest.approx(oracle.chi2(maps, target, 0.5), rel=1e-5)
        ref, _ = fd_reference(base, lambda m: oracle.chi2(m, target, 0.5), pix=pix)
        assert_grad(grad.cpu().numpy(), ref, what=f"chi2 Nside {base.nside}, N {base.n_steps}, pixels {begin}+{count}")


@pytest.mark.slow
def test_vjp_full_size_sampled(torch):
    """Nside 64, 512 steps, 4 frequencies, 16 parameters (the adjoint workload),
    with seeds on 120 sampled pixels so the FD reference needs only those."""
    prob = inputs.config2()
    pix = inputs.sample_pixels(prob.npix, 120, seed=31)
    gm = seeds(prob, seed=9, pix=pix)
    g = adjoint(prob, gmaps=torch.tensor(gm, dtype=torch.float32, device="cuda")).cpu().numpy()
    gsub = gm[:, :, pix]
    ref, _ = fd_reference(prob, lambda m: float(np.sum(gsub * m)), pix=pix)
    assert_grad(g, ref, what="full-size VJP")


@pytest.mark.slow
def test_chi2_full_size_value(torch):
    """chi^2 of the full Nside-64 map against an oracle-rendered target."""
    prob, th_target, sigma = inputs.config3()
    target = oracle.forward(prob.with_theta(th_target))
    target = target + inputs.target_noise(target.shape, seed=3, sigma=sigma)
    grad, chi2 = adjoint(prob, target=torch.tensor(target, dtype=torch.float32, device="cuda"),
                         sigma=sigma)
    chi2_ora = oracle.chi2(oracle.forward(prob), target, sigma)
    assert float(chi2.item()) == pytest.approx(chi2_ora, rel=1e-5)
    assert np.all(np.isfinite(grad.cpu().numpy()))


def test_deterministic_and_streams(torch):
    prob, target, sigma = chi2_problem(4, 96)
    tt = torch.tensor(target, dtype=torch.float32, device="cuda")
    a, ca = adjoint(prob, target=tt, sigma=sigma)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b, cb = adjoint(prob, target=tt, sigma=sigma)
    s.synchronize()
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    assert float(ca.item()) == float(cb.item())


def test_autograd_function(torch):
    prob = inputs.config2().replace(nside=4, n_steps=64)
    theta = torch.tensor(prob.theta, dtype=torch.float64, requires_grad=True)
    maps = SynaxMaps.apply(theta, prob)
    gm = torch.tensor(seeds(prob, seed=12), dtype=torch.float32, device="cuda")
    loss = (maps * gm).sum()
    loss.backward()
    direct = adjoint(prob, gmaps=gm).cpu().numpy()
    assert np.array_equal(theta.grad.numpy(), direct)


def test_empty_range_and_pixel_range(torch):
    prob = inputs.config2().replace(nside=4, n_steps=64)
    empty = prob.replace(pix_begin=prob.npix)
    z = torch.zeros((4, 3, 0), device="cuda")
    g = adjoint(empty, gmaps=z).cpu().numpy()
    assert np.all(g == 0)
    # a pixel range gives the gradient of that range's seeds
    part = prob.replace(pix_begin=40, pix_count=60)
    gm = seeds(part, seed=5)
    g_part = adjoint(part, gmaps=torch.tensor(gm, device="cuda", dtype=torch.float32)).cpu().numpy()
    full = np.zeros((4, 3, prob.npix))
    full[:, :, 40:100] = gm
    g_full = adjoint(prob, gmaps=torch.tensor(full, device="cuda", dtype=torch.float32)).cpu().numpy()
    assert np.allclose(g_part, g_full, rtol=1e-5, atol=1e-6 * np.abs(g_full).max())
