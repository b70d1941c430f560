"""The persistent, graph-captured batch (synax_batch_*) against the FP64
oracle and against one-map synax_adjoint calls on the same sets.

Against the oracle: every set's chi^2 gradient (Eq. 15) and VJP gradient
against Richardson-extrapolated central differences of the oracle (h and h/2,
h_i = 1e-4 s_i), per component |g - g_FD| <= 1e-3 |g_FD| + 1e-4 max |g_FD|,
the adjoint tests' tolerance; maps to the stated I and Q/U tolerances.

Against the one-map call: the batch runs the same per-CTA adjoint code,
inlined into another kernel and with its own lanes-per-ray width per set, so
per-ray FP32 rounding may differ: gradients are compared at FP32 precision
(1e-5 relative, 1e-6 of the largest component), bitwise only between replays."""
import numpy as np
import pytest

import oracle
from paper_2410_01136_gb300 import BatchPlan, adjoint, forward, inputs

from .parity import assert_parity, assert_parity_coarse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_01136_gb300 import build
    build()
    oracle.build()
    return _t


def small_sets(n=10, seed=4):
    sets = inputs.config4(n_sets=n, seed=seed)
    nsides = (2, 4, 8)
    steps = (32, 64, 100, 128)
    return [s.replace(nside=nsides[i % 3], n_steps=steps[i % 4]) for i, s in enumerate(sets)]


def targets_for(torch, sets, seed=3):
    out = []
    for i, p in enumerate(sets):
        th = inputs.perturbed_theta(p.theta, seed=seed + i)
        t = oracle.forward(p.with_theta(th)) + inputs.target_noise((p.n_freq, 3, p.npix), seed=seed + i)
        out.append(torch.tensor(t, dtype=torch.float32, device="cuda"))
    return out


def fd_chi2_reference(prob, target, sigma):
    """Richardson-extrapolated central differences of the oracle's chi^2."""
    th = prob.theta
    h = 1e-4 * inputs.jf12_scales(th)

    def L(t):
        return oracle.chi2(oracle.forward(prob.with_theta(t)), target, sigma)
    g1 = oracle.fd_gradient(L, th, h)
    g2 = oracle.fd_gradient(L, th, h / 2)
    return (4 * g2 - g1) / 3


def fd_vjp_reference(prob, seed):
    th = prob.theta
    h = 1e-4 * inputs.jf12_scales(th)

    def L(t):
        return float(np.sum(seed * oracle.forward(prob.with_theta(t))))
    g1 = oracle.fd_gradient(L, th, h)
    g2 = oracle.fd_gradient(L, th, h / 2)
    return (4 * g2 - g1) / 3


def chi2_tolerance(ora, target, sigma, freqs, n_steps):
    """Bound on |chi^2 - chi^2_oracle| implied by maps at the stated
    tolerances: every entry may differ from the oracle by b_e (1e-5 |I|;
    1e-4 max(|P|, 1e-2 median |P|) for Q and U, 2e-4 below 1 GHz for
    marches of fewer than 16 steps), so chi^2 moves by at most
    sum (2 |M - T| b_e + b_e^2) / sigma^2."""
    b = np.empty_like(ora)
    for f, nu in enumerate(freqs):
        b[f, 0] = 1e-5 * np.abs(ora[f, 0])
        P = np.hypot(ora[f, 1], ora[f, 2])
        tol = 2e-4 if (n_steps < 16 and nu < 1e9) else 1e-4
        bp = tol * np.maximum(P, 1e-2 * np.median(P))
        b[f, 1] = bp
        b[f, 2] = bp
    return float(np.sum(2 * np.abs(ora - target) * b + b * b)) / sigma ** 2


def assert_grad(g, ref, what, rel=1e-3, floor=1e-4):
    g = np.asarray(g, dtype=np.float64)
    tol = rel * np.abs(ref) + floor * np.max(np.abs(ref))
    bad = np.where(np.abs(g - ref) > tol)[0]
    assert bad.size == 0, (what, [(int(i), float(g[i]), float(ref[i])) for i in bad])


def mixed_sets():
    """Six sets of the ensemble draw at Nside 2-8 and 13-128 steps: the step
    counts fall in different lanes-per-ray bins, 13 leaves lane chunks of one
    or two samples, and two sets share a size but not their parameters."""
    sets = inputs.config4(n_sets=6, seed=11)
    shapes = [(2, 13), (4, 128), (8, 64), (2, 100), (8, 37), (4, 128)]
    return [s.replace(nside=n, n_steps=k) for s, (n, k) in zip(sets, shapes)]


def test_batch_gradient_against_oracle(torch):
    sets = mixed_sets()
    sigma = 0.5
    tg_np = []
    for i, p in enumerate(sets):
        th = inputs.perturbed_theta(p.theta, seed=30 + i)
        tg_np.append(oracle.forward(p.with_theta(th)) + inputs.target_noise((p.n_freq, 3, p.npix), seed=30 + i))
    tg = [torch.tensor(t, dtype=torch.float32, device="cuda") for t in tg_np]
    plan = BatchPlan(sets)
    maps = [torch.empty_like(t) for t in tg]
    grads, chi2 = plan.run(targets=tg, sigma=sigma, maps=maps)
    g = grads.cpu().numpy()
    c = chi2.cpu().numpy()
    for i, p in enumerate(sets):
        ora = oracle.forward(p)
        if p.n_steps < 16:
            assert_parity_coarse(maps[i].cpu().numpy(), ora, p.freq_hz, f"batch set {i} maps")
        else:
            assert_parity(maps[i].cpu().numpy(), ora, what=f"batch set {i} maps")
        c_ora = oracle.chi2(ora, tg_np[i], sigma)
        assert abs(c[i] - c_ora) <= chi2_tolerance(ora, tg_np[i], sigma, p.freq_hz, p.n_steps), (i, c[i], c_ora)
        assert_grad(g[i], fd_chi2_reference(p, tg_np[i], sigma), f"batch set {i} chi2 gradient")
    # VJP mode of the same plan, two sets against the oracle
    seeds_np = [inputs.normal(inputs.substream(80 + i, p.npix), p.n_freq * 3 * p.npix).reshape(p.n_freq, 3, p.npix)
                for i, p in enumerate(sets)]
    gv, _ = plan.run(seeds=[torch.tensor(s, dtype=torch.float32, device="cuda") for s in seeds_np])
    gv = gv.cpu().numpy()
    for i in (1, 4):
        assert_grad(gv[i], fd_vjp_reference(sets[i], seeds_np[i]), f"batch set {i} VJP gradient")
    plan.close()


def test_batch_matches_single_adjoint(torch):
    sets = small_sets()
    tg = targets_for(torch, sets)
    plan = BatchPlan(sets)
    maps = [torch.empty_like(t) for t in tg]
    grads, chi2 = plan.run(targets=tg, sigma=0.5, maps=maps)
    torch.cuda.synchronize()
    g = grads.cpu().numpy()
    c = chi2.cpu().numpy()
    for i, p in enumerate(sets):
        gi, ci = adjoint(p, target=tg[i], sigma=0.5)
        gi = gi.cpu().numpy()
        assert np.allclose(g[i], gi, rtol=1e-5, atol=1e-6 * np.abs(gi).max()), i
        assert c[i] == pytest.approx(float(ci.item()), rel=1e-6)
        # the same arithmetic compiled into another kernel (another register
        # budget, so FMA contraction may differ): I to rounding, Q+iU (which
        # cancels by up to ~100x at 408 MHz) to 1e-5
        assert_parity(maps[i].cpu().numpy(), forward(p).cpu().numpy(), 1e-6, 1e-5, f"set {i} maps")
        # chi^2 against the oracle's maps
        ora = oracle.chi2(oracle.forward(p), tg[i].cpu().numpy(), 0.5)
        assert c[i] == pytest.approx(ora, rel=1e-5)
    lat = plan.latencies()
    assert np.all(np.isfinite(lat)) and np.all(lat >= 0)
    info = plan.info()
    assert info["n_tiles"] > 0 and info["grid"] > 0
    plan.close()


def test_graph_replay_new_thetas_and_vjp(torch):
    sets = small_sets(6, seed=9)
    tg = targets_for(torch, sets, seed=20)
    plan = BatchPlan(sets)
    g0, _ = plan.run(targets=tg, sigma=0.5)
    g0 = g0.cpu().numpy()
    g0b, _ = plan.run(targets=tg, sigma=0.5)            # replay, same inputs: bitwise equal
    assert np.array_equal(g0, g0b.cpu().numpy())
    new = np.stack([inputs.perturbed_theta(p.theta, seed=50 + i, frac=0.02) for i, p in enumerate(sets)])
    new[:, 13] = np.clip(new[:, 13], 2.8, 3.2)
    g1, c1 = plan.run(targets=tg, sigma=0.5, thetas=new)
    g1 = g1.cpu().numpy()
    for i, p in enumerate(sets):
        gi, ci = adjoint(p.with_theta(new[i]), target=tg[i], sigma=0.5)
        assert np.allclose(g1[i], gi.cpu().numpy(), rtol=1e-5, atol=1e-6 * np.abs(g1[i]).max())
    # VJP mode through the same plan (new graph launch, same descriptors layout)
    seeds = [torch.tensor(inputs.normal(70 + i, p.n_freq * 3 * p.npix).reshape(p.n_freq, 3, p.npix),
                          dtype=torch.float32, device="cuda") for i, p in enumerate(sets)]
    gv, cv = plan.run(seeds=seeds)
    assert cv is None
    gv = gv.cpu().numpy()
    for i, p in enumerate(sets):
        ref = adjoint(p.with_theta(new[i]), gmaps=seeds[i]).cpu().numpy()
        assert np.allclose(gv[i], ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())
    plan.close()


@pytest.mark.slow
def test_ensemble_workload_subset(torch):
    """16 sets of the 256-set ensemble draw (Nside 16-128, 128-1024 steps)."""
    sets = inputs.config4()[:16]
    tg = [forward(p.with_theta(inputs.perturbed_theta(p.theta, seed=5 + i))).contiguous()
          for i, p in enumerate(sets)]
    plan = BatchPlan(sets)
    grads, chi2 = plan.run(targets=tg, sigma=0.5)
    g = grads.cpu().numpy()
    for i, p in enumerate(sets):
        gi, _ = adjoint(p, target=tg[i], sigma=0.5)
        gi = gi.cpu().numpy()
        assert np.allclose(g[i], gi, rtol=1e-5, atol=1e-6 * np.abs(gi).max()), i
    lat = plan.latencies()
    assert np.all(lat > 0)
    plan.close()


def test_plan_validation(torch):
    from paper_2410_01136_gb300 import SynaxError
    a = inputs.config2().replace(nside=2, n_steps=16)
    with pytest.raises(SynaxError):
        BatchPlan([a, a.replace(freq_hz=(1e9,))])             # mixed frequency counts
    with pytest.raises(SynaxError):
        BatchPlan([a.replace(f64=True)])                       # FP64 batch
    with pytest.raises(SynaxError):
        BatchPlan([inputs.toy_problem(nside=2, n_steps=8)])     # no adjoint for the toy
