"""The device-resident batch and the HMC sampler (synax_batch_bind /
synax_batch_run_device, synax_hmc_*) on the GPU.

- run_device with theta on the device gives the gradients and chi^2 of the
  host-theta run (the parameter-dependent constants come from the same code
  on the device);
- the sampler's trajectory equals the oracle's HMC (oracle/hmc.py: same
  algorithm, same documented random numbers, chi^2 and gradient from the
  FP64 oracle with Richardson-extrapolated central differences): every
  accept decision and every draw, to the gradient's FP32 accuracy;
- a warmed-up ensemble accepts at a usable rate and its chains mix.
"""
import numpy as np
import pytest

import oracle
from oracle import hmc as ohmc
from paper_2410_01136_gb300 import HMC, BatchPlan, effective_sample_size, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_01136_gb300 import build
    build()
    oracle.build()
    return _t


def test_run_device_matches_host_run(torch):
    sets = [inputs.config2().replace(nside=n, n_steps=s) for n, s in ((8, 64), (16, 100), (8, 128))]
    thetas = np.stack([inputs.perturbed_theta(p.theta, seed=80 + i) for i, p in enumerate(sets)])
    targets = [torch.tensor(oracle.forward(p.with_theta(inputs.perturbed_theta(p.theta, seed=90 + i))),
                            dtype=torch.float32, device="cuda") for i, p in enumerate(sets)]
    plan = BatchPlan(sets)
    g_host, c_host = plan.run(targets=targets, sigma=0.5, thetas=thetas)
    g_host, c_host = g_host.clone(), c_host.clone()
    plan2 = BatchPlan(sets)
    g_dev, c_dev = plan2.bind(targets=targets, sigma=0.5)
    plan2.run_device(torch.tensor(thetas, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    np.testing.assert_allclose(c_dev.cpu().numpy(), c_host.cpu().numpy(), rtol=1e-6)
    np.testing.assert_allclose(g_dev.cpu().numpy(), g_host.cpu().numpy(), rtol=1e-5,
                               atol=1e-6 * np.abs(g_host.cpu().numpy()).max())
    plan.close()
    plan2.close()


FREE = [0, 1, 2, 3]          # b0, psi0, psi1, chi0B of the WMAP-type model (Sec. 3.2 samples these four)


def small_wmap():
    th = inputs.wmap_theta()
    th[2], th[3] = 0.05, 0.3
    return inputs.Problem(nside=2, n_steps=32, freq_hz=(1.4e9, 2.4e9), model_id=inputs.MODEL_WMAP, theta=th)


def oracle_chi2_grad(prob, target, sigma):
    def f(thetas):
        c2 = np.empty(len(thetas))
        g = np.zeros_like(thetas)
        for c, th in enumerate(thetas):
            def L(t):
                return oracle.chi2(oracle.forward(prob.with_theta(t)), target, sigma)
            c2[c] = L(th)
            for j in FREE:
                h = 1e-4 * max(abs(th[j]), 1e-2)
                e = np.zeros_like(th)
                e[j] = 1.0
                d1 = (L(th + h * e) - L(th - h * e)) / (2 * h)
                d2 = (L(th + 0.5 * h * e) - L(th - 0.5 * h * e)) / h
                g[c, j] = (4 * d2 - d1) / 3
        return c2, g
    return f


def test_hmc_matches_oracle(torch):
    prob = small_wmap()
    sigma = 0.05
    truth = prob.theta.copy()
    truth[FREE] *= 1.02
    target = oracle.forward(prob.with_theta(truth))
    target = target + inputs.target_noise(target.shape, seed=81, sigma=sigma)
    C = 3
    th0 = np.stack([prob.theta * (1.0 + 0.01 * inputs.normal(inputs.substream(82, c), prob.theta.size)
                                  * np.isin(np.arange(prob.theta.size), FREE)) for c in range(C)])
    inv_mass = np.zeros(prob.theta.size)
    inv_mass[FREE] = (0.01 * np.maximum(np.abs(prob.theta[FREE]), 0.05)) ** 2
    eps, L, seed = 0.6, 3, 1234
    tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
    hmc = HMC([prob.with_theta(t) for t in th0], [tgt] * C, sigma, th0, eps, L, seed=seed, inv_mass=inv_mass)
    draws, acc = hmc.run(4)
    torch.cuda.synchronize()
    ref_draws, ref_acc = ohmc.hmc_iterations(th0, oracle_chi2_grad(prob, target, sigma), 4, eps, L, seed, inv_mass)
    np.testing.assert_array_equal(acc.cpu().numpy(), ref_acc)
    assert 0 < ref_acc.sum() < ref_acc.size or ref_acc.all()
    d = draws.cpu().numpy()
    scale = np.sqrt(np.where(inv_mass > 0, inv_mass, 1.0))
    np.testing.assert_allclose(d / scale, ref_draws / scale, rtol=0, atol=1e-3)
    fixed = np.setdiff1d(np.arange(prob.theta.size), FREE)
    np.testing.assert_array_equal(d[:, :, fixed], np.broadcast_to(th0[None, :, fixed], d[:, :, fixed].shape))
    hmc.close()


def test_warmed_up_ensemble_mixes(torch):
    prob = small_wmap().replace(nside=4, n_steps=64)
    sigma = 0.05
    target = oracle.forward(prob) + inputs.target_noise((2, 3, prob.npix), seed=83, sigma=sigma)
    C = 32
    th0 = np.repeat(prob.theta[None, :], C, axis=0)
    inv_mass = np.zeros(prob.theta.size)
    inv_mass[FREE] = (0.01 * np.maximum(np.abs(prob.theta[FREE]), 0.05)) ** 2
    tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
    hmc = HMC([prob] * C, [tgt] * C, sigma, th0, 0.3, 6, seed=7, inv_mass=inv_mass)
    hmc.warmup(60)
    draws, acc = hmc.run(60)
    a = float(acc.float().mean().item())
    assert 0.3 < a < 0.98, a
    d = draws.cpu().numpy()
    ess = effective_sample_size(d[:, :, FREE])
    assert np.all(ess > 10), ess           # correlated psi0, psi1, chi0B mix slower under a diagonal mass
    assert np.all(d[:, :, 4:] == th0[0, 4:])
    hmc.close()


def test_error_paths(torch):
    from paper_2410_01136_gb300 import SynaxError, _native
    prob = small_wmap()
    plan = BatchPlan([prob, prob])
    th = torch.tensor(np.stack([prob.theta, prob.theta]), dtype=torch.float64, device="cuda")
    with pytest.raises(SynaxError) as e:
        plan.run_device(th)                              # not bound
    assert e.value.status == _native.SYNAX_EINVAL
    tgt = torch.zeros((2, 3, prob.npix), dtype=torch.float32, device="cuda")
    with pytest.raises(SynaxError):
        plan.bind(targets=[tgt, tgt], sigma=0.0)
    with pytest.raises(SynaxError) as e:
        plan.bind(targets=[tgt, tgt], sigma=float("nan"))
    assert e.value.status == _native.SYNAX_ENONFINITE
    plan.close()
    th0 = np.stack([prob.theta, prob.theta])
    for kw in (dict(step_size=0.0, n_leapfrog=2), dict(step_size=0.1, n_leapfrog=0),
               dict(step_size=0.1, n_leapfrog=2, inv_mass=-np.ones(8)),
               dict(step_size=0.1, n_leapfrog=2, lo=np.ones(8), hi=np.zeros(8))):
        with pytest.raises(SynaxError):
            HMC([prob, prob], [tgt, tgt], 0.05, th0, **kw)
    bad = th0.copy()
    bad[1, 0] = np.nan
    with pytest.raises(SynaxError) as e:
        HMC([prob, prob], [tgt, tgt], 0.05, bad, 0.1, 2)
    assert e.value.status == _native.SYNAX_ENONFINITE
    hmc = HMC([prob, prob], [tgt, tgt], 0.05, th0, 0.1, 2)
    with pytest.raises(SynaxError):
        hmc.set(step_size=-1.0)
    hmc.close()
