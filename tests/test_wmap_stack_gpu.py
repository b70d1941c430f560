"""The stacked WMAP model of Sec. 4.3 (Eq. 16) on the GPU against the FP64
oracle, through the C ABI: maps (FP32 and FP64, 408 MHz to 2.4 GHz, to the
stated tolerances, tests/parity.py), the full Nside-64 workload at sampled
pixels, fields at
points, and the 19-component gradient (16 field parameters of the paper's
table + N0_obs, p, n_e0) against Richardson-extrapolated central
differences of the oracle, as in tests/test_adjoint_gpu.py."""
import numpy as np
import pytest

import oracle
from paper_2410_01136_gb300 import adjoint, eval_fields, forward, grid_sample, inputs

from .parity import assert_parity, assert_parity_by_frequency

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_01136_gb300 import build
    build()
    oracle.build()
    return _t


def small(f64=False, nside=8, n_steps=100, freqs=(408e6, 1.4e9, 2.4e9), **kw):
    return inputs.wmap_stack_problem(nside=nside, n_steps=n_steps, freq_hz=freqs, f64=f64, **kw)


@pytest.mark.parametrize("f64", [False, True])
@pytest.mark.parametrize("kw", [dict(), dict(pix_begin=51, pix_count=600, n_steps=77),
                                dict(box_clip=False, r_max_kpc=20.0, obs_kpc=inputs.OBS_CONFIG_KPC)])
def test_forward_parity(torch, f64, kw):
    prob = small(f64, **kw)
    m = forward(prob).cpu().numpy()
    ref = oracle.forward(prob, pix=np.arange(prob.pix_begin, prob.pix_begin + prob.n_pix_out))
    assert_parity_by_frequency(m, ref, prob.freq_hz, f64, "stacked WMAP")


def test_forward_full_size_sampled(torch):
    prob = inputs.wmap_stack_problem()                 # Nside 64, 512 steps, 2.4 GHz, box
    m = forward(prob).cpu().numpy()
    pix = inputs.sample_pixels(prob.npix, 96, seed=14)
    assert_parity(m[:, :, pix], oracle.forward(prob, pix=pix), what="stacked WMAP full size")


def test_forward_full_size_sampled_408mhz(torch):
    prob = inputs.wmap_stack_problem(freq_hz=(408e6,))
    m = forward(prob).cpu().numpy()
    pix = inputs.sample_pixels(prob.npix, 96, seed=16)
    assert_parity(m[:, :, pix], oracle.forward(prob, pix=pix), what="stacked WMAP full size 408 MHz")


@pytest.mark.parametrize("f64", [False, True])
def test_fields_and_grid_sample(torch, f64):
    prob = small(f64)
    u = inputs.uniform(inputs.substream(70, 1), 3 * 300, -0.5, 0.5).reshape(300, 3)
    pos = u * np.asarray(prob.box_kpc)
    out = eval_fields(prob, pos, np.zeros(300)).cpu().numpy()
    ref = np.array([np.concatenate([oracle.fields(prob, r)[0], oracle.fields(prob, r)[1:]]) for r in pos])
    scale = np.abs(ref[:, :3]).max()
    np.testing.assert_allclose(out[:, :3], ref[:, :3], rtol=0, atol=(1e-12 if f64 else 2e-6) * scale)
    np.testing.assert_allclose(out[:, 3:], ref[:, 3:], rtol=1e-12 if f64 else 1e-5)
    g = grid_sample(prob, (8, 6, 5)).cpu().numpy().reshape(-1, 3)        # no node on the z axis
    x, y, z = (np.linspace(-0.5 * prob.box_kpc[a], 0.5 * prob.box_kpc[a], n) for a, n in enumerate((8, 6, 5)))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    nodes = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)
    gref = np.array([oracle.fields(prob, r)[0] for r in nodes])
    np.testing.assert_allclose(g, gref, rtol=0, atol=(1e-12 if f64 else 2e-6) * np.abs(gref).max())


def fd_reference(prob, loss, h_rel=1e-4):
    th = prob.theta
    h = h_rel * np.abs(th)

    def L(t):
        return loss(oracle.forward(prob.with_theta(t)))
    g1 = oracle.fd_gradient(L, th, h)
    g2 = oracle.fd_gradient(L, th, h / 2)
    return (4 * g2 - g1) / 3


def assert_grad(g, ref, rel, floor, what):
    g = np.asarray(g, dtype=np.float64)
    tol = rel * np.abs(ref) + floor * np.max(np.abs(ref))
    bad = np.where(np.abs(g - ref) > tol)[0]
    assert bad.size == 0, (what, [(int(i), float(g[i]), float(ref[i])) for i in bad])


@pytest.mark.parametrize("f64", [False, True])
def test_vjp_gradient(torch, f64):
    prob = small(f64, nside=4, n_steps=64)
    n = prob.n_pix_out
    gm = inputs.normal(inputs.substream(71, n), prob.n_freq * 3 * n).reshape(prob.n_freq, 3, n)
    dt = torch.float64 if f64 else torch.float32
    g = adjoint(prob, gmaps=torch.tensor(gm, dtype=dt, device="cuda")).cpu().numpy()
    assert g.shape == (19,)
    ref = fd_reference(prob, lambda m: float(np.sum(gm * m)))
    if f64:
        assert_grad(g, ref, 1e-6, 1e-7, "stacked WMAP VJP FP64")
    else:
        assert_grad(g, ref, 1e-3, 1e-4, "stacked WMAP VJP FP32")


def test_chi2_gradient_at_2400mhz(torch):
    """Sec. 4.3's likelihood: Q/U (and I) at 2.4 GHz against a noisy mock."""
    prob = small(nside=8, n_steps=128, freqs=(2.4e9,))
    truth = prob.with_theta(prob.theta * (1.0 + 0.03 * inputs.normal(inputs.substream(72, 1), 19)))
    target = oracle.forward(truth)
    target = target + inputs.target_noise(target.shape, seed=73, sigma=1e-3)
    grad, chi2 = adjoint(prob, target=torch.tensor(target, dtype=torch.float32, device="cuda"), sigma=1e-3)
    ref = fd_reference(prob, lambda m: oracle.chi2(m, target, 1e-3))
    assert float(chi2.item()) == pytest.approx(oracle.chi2(oracle.forward(prob), target, 1e-3), rel=1e-4)
    assert_grad(grad.cpu().numpy(), ref, 1e-3, 1e-4, "stacked WMAP chi2")
