"""The learned surrogate's CUDA path against the FP64 oracle (oracle/surrogate.py).

Precision: the kernels round GEMM operands (inputs, weights, activations,
output gradients) to BF16 and accumulate in FP32; the oracle rounds the same
values at the same points and sums in FP64.  What remains is FP32 versus
FP64 summation (~1e-6 relative) plus occasional one-ulp BF16 flips where a
value sits at a rounding boundary (2^-8 relative on that element), so tensors
are compared norm-wise at 4e-3 and element-wise at 2e-2 of the largest entry.
"""
import math

import numpy as np
import pytest

from oracle import surrogate as so
from paper_2410_01136_gb300 import inputs

pytestmark = pytest.mark.gpu

NORM_TOL = 4e-3
ELEM_TOL = 2e-2


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_01136_gb300 import build
    build()
    return _t


def small(torch, n_theta=5, width=128, depth=2, nside=4, n_basis=64, batch=64, seed=1, **kw):
    from paper_2410_01136_gb300.surrogate import Surrogate
    lo = -1.0 - np.arange(n_theta) * 0.5
    hi = 2.0 + np.arange(n_theta)
    sign, rows = inputs.surrogate_basis_spec(nside, n_basis, seed=seed)
    sur = Surrogate(n_theta, lo, hi, sign, rows, width=width, depth=depth, nside=nside, batch=batch, **kw)
    rng = np.random.default_rng(seed)
    params = []
    for l in range(len(sur.widths) - 1):
        k, n = sur.widths[l], sur.widths[l + 1]
        params.append(((rng.normal(size=(n, k)) * 1.5 / math.sqrt(k)).astype(np.float32),
                       (rng.normal(size=n) * 0.1).astype(np.float32)))
    sur.set_params(params)
    return sur, params, lo, hi, sign, rows


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def assert_close(got, ref, what):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    r = rel(got, ref)
    e = float(np.max(np.abs(got - ref))) / max(float(np.max(np.abs(ref))), 1e-300)
    assert r <= NORM_TOL and e <= ELEM_TOL, f"{what}: norm-wise {r:.3e}, element-wise {e:.3e}"


@pytest.mark.parametrize("nside,n_basis,n_maps", [(4, 64, 5), (8, 128, 7), (8, 768, 2)])
def test_projection_matches_oracle(torch, nside, n_basis, n_maps):
    sur, _, _, _, sign, rows = small(torch, nside=nside, n_basis=n_basis, map_chunk=2)
    N = 12 * nside * nside
    rng = np.random.default_rng(nside + n_basis)
    maps = (50.0 + 20.0 * rng.normal(size=(n_maps, 3, N))).astype(np.float32)
    c = sur.project(torch.tensor(maps, device="cuda")).cpu().numpy()
    ref = so.project(maps.astype(np.float64), nside, sign, rows)
    scale = np.linalg.norm(maps.astype(np.float64), axis=-1, keepdims=True)
    assert np.max(np.abs(c - ref) / scale) < 2e-6
    sur.status()
    sur.close()


def test_projection_full_size_sampled(torch):
    """Nside 64, 3072 basis vectors: sampled coefficients of a seeded map."""
    from paper_2410_01136_gb300.surrogate import Surrogate
    sign, rows = inputs.surrogate_basis_spec(64, 3072, seed=5)
    lo, hi = inputs.config5_box()
    sur = Surrogate(16, lo, hi, sign, rows, width=64, depth=1, nside=64, batch=64, max_eval=64, map_chunk=4)
    N = 49152
    rng = np.random.default_rng(3)
    maps = (30.0 + 10.0 * rng.normal(size=(2, 3, N))).astype(np.float32)
    c = sur.project(torch.tensor(maps, device="cuda")).cpu().numpy()
    pick = inputs.sample_pixels(3072, 48, seed=8)
    ref = so.project(maps.astype(np.float64), 64, sign, rows[pick])
    scale = np.linalg.norm(maps.astype(np.float64), axis=-1, keepdims=True)
    assert np.max(np.abs(c[..., pick] - ref) / scale) < 2e-6
    sur.close()


def _batch(torch, sur, lo, hi, seed, n=None):
    rng = np.random.default_rng(seed)
    n = n or sur.batch
    theta = (lo + (hi - lo) * rng.uniform(size=(n, sur.n_theta))).astype(np.float32)
    coeff = (3.0 * rng.normal(size=(n, sur.n_out)) + 1.0).astype(np.float32)
    return theta, coeff


def test_step_loss_and_gradients_match_oracle(torch):
    sur, params, lo, hi, _, _ = small(torch)
    mean = np.linspace(-1, 1, sur.n_out).astype(np.float32)
    scale = 2.5
    sur.set_normalization(mean, scale)
    theta, coeff = _batch(torch, sur, lo, hi, 11)
    loss = sur.step(torch.tensor(theta, device="cuda"), torch.tensor(coeff, device="cuda"), update=False)
    loss = float(loss.item())
    g = sur.grads()
    x = so.normalize_theta(theta.astype(np.float64), lo, hi)
    y = (coeff.astype(np.float64) - mean) / scale
    ref_loss, ref_g = so.mse_loss_and_grads([(W.astype(np.float64), b.astype(np.float64)) for W, b in params],
                                            x, y, bf16=True)
    assert abs(loss - ref_loss) <= 2e-3 * ref_loss
    for l, ((gw, gb), (rw, rb)) in enumerate(zip(g, ref_g)):
        assert_close(gw, rw, f"dW{l}")
        assert_close(gb, rb, f"db{l}")
    # without the BF16 rounding the oracle is the exact gradient: the kernels
    # stay within BF16 distance of it
    _, exact = so.mse_loss_and_grads([(W.astype(np.float64), b.astype(np.float64)) for W, b in params], x, y,
                                     bf16=False)
    for (gw, _), (ew, _) in zip(g, exact):
        assert rel(gw, ew) < 5e-2
    sur.close()


def test_adam_update_matches_oracle(torch):
    lr = 3e-3
    sur, params, lo, hi, _, _ = small(torch, lr=lr, lr_min=1e-4, total_steps=50)
    theta, coeff = _batch(torch, sur, lo, hi, 12)
    th = torch.tensor(theta, device="cuda")
    cf = torch.tensor(coeff, device="cuda")
    sur.step(th, cf, update=False)
    g = sur.grads()
    sur.step(th, cf, update=True)                      # same batch: the same gradient
    g2 = sur.grads()
    for (a, b), (c, d) in zip(g, g2):
        assert np.array_equal(a, c) and np.array_equal(b, d), "gradient is not deterministic"
    new = sur.params()
    m1, v1 = sur.adam_moments()
    for (W, b), (gw, gb), (nw, nb), (mw, mb) in zip(params, g, new, m1):
        for w0, gg, w1, mm in ((W, gw, nw, mw), (b, gb, nb, mb)):
            ref_w, ref_m, ref_v = so.adam_step(w0.astype(np.float64), gg.astype(np.float64), 0.0, 0.0, 1,
                                               lr=so.cosine_lr(0, lr, 1e-4, 50))
            assert np.max(np.abs(w1 - ref_w)) <= 1e-6 * np.max(np.abs(w0)) + 1e-3 * lr
            assert np.allclose(mm, ref_m, rtol=1e-6, atol=1e-12)
    # a second step uses t = 2 and the schedule's second rate
    sur.step(th, cf, update=True)
    g3 = sur.grads()
    new2 = sur.params()
    m2, v2 = sur.adam_moments()
    for (w1, b1), (gw, gb), (w2, b2), (mw, mb), (vw, vb) in zip(new, g3, new2, m1, v1):
        ref_w, _, _ = so.adam_step(w1.astype(np.float64), gw.astype(np.float64), mw, vw, 2,
                                   lr=so.cosine_lr(1, lr, 1e-4, 50))
        assert np.max(np.abs(w2 - ref_w)) <= 1e-6 * np.max(np.abs(w1)) + 1e-3 * lr
    sur.close()


@pytest.mark.parametrize("width", [128, 320])
def test_eval_and_vjp_match_oracle(torch, width):
    """Width 320 takes the 128-column GEMM tiles whose GELU and GELU' epilogues
    stage their BF16 outputs for TMA stores (three column tiles, the last one
    half full; 50-row chunks leave the row tile ragged)."""
    sur, params, lo, hi, _, _ = small(torch, width=width, max_eval=50)      # 3 chunks for n = 130
    mean = np.linspace(2, -2, sur.n_out).astype(np.float32)
    scale = 1.7
    sur.set_normalization(mean, scale)
    theta, _ = _batch(torch, sur, lo, hi, 13, n=130)
    gc = np.random.default_rng(14).normal(size=(130, sur.n_out)).astype(np.float32)
    th = torch.tensor(theta, device="cuda")
    c_only = sur(th).cpu().numpy().reshape(130, -1)
    c, gt = sur(th, torch.tensor(gc, device="cuda").reshape(130, 3, -1))
    c = c.cpu().numpy().reshape(130, -1)
    gt = gt.cpu().numpy()
    assert np.array_equal(c, c_only)
    # a seed 4 bytes off a 16-byte boundary takes the scalar seed conversion:
    # the same numbers
    buf = torch.zeros(130 * sur.n_out + 1, device="cuda")
    buf[1:] = torch.tensor(gc, device="cuda").reshape(-1)
    _, gt_odd = sur(th, buf[1:].reshape(130, 3, -1))
    assert np.array_equal(gt_odd.cpu().numpy(), gt)
    P = [(W.astype(np.float64), b.astype(np.float64)) for W, b in params]
    x = so.normalize_theta(theta.astype(np.float64), lo, hi)
    zs, xs = so.mlp_forward(P, x, bf16=True)
    ref_c = mean + scale * zs[-1]
    assert_close(c - mean, ref_c - mean, "coefficients")
    _, dx = so.mlp_backward(P, zs, xs, so.bf16_round(gc.astype(np.float64) * scale), bf16=True)
    ref_gt = dx * (2.0 / (hi - lo))[None, :]
    assert_close(gt, ref_gt, "dL/dtheta")
    sur.close()


def test_vjp_matches_finite_differences_of_surrogate(torch):
    """The surrogate's own gradient against central differences of its own
    forward (FP32 evaluation of a smooth function): a check that the VJP is
    the derivative of what the forward computes."""
    sur, params, lo, hi, _, _ = small(torch, width=64, depth=1)
    sur.set_normalization(np.zeros(sur.n_out, np.float32), 1.0)
    P = [(W.astype(np.float64), b.astype(np.float64)) for W, b in params]
    theta = ((lo + hi) / 2 + 0.1 * (hi - lo)).astype(np.float64)[None, :]
    gc = np.random.default_rng(4).normal(size=(1, sur.n_out))
    _, gt = sur(torch.tensor(theta, dtype=torch.float32, device="cuda"),
                torch.tensor(gc, dtype=torch.float32, device="cuda").reshape(1, 3, -1))
    gt = gt.cpu().numpy()[0]
    fd = np.empty(sur.n_theta)
    for j in range(sur.n_theta):
        h = 1e-3 * (hi[j] - lo[j])
        tp, tm = theta.copy(), theta.copy()
        tp[0, j] += h
        tm[0, j] -= h
        fp = so.mlp_forward(P, so.normalize_theta(tp, lo, hi), bf16=False)[0][-1]
        fm = so.mlp_forward(P, so.normalize_theta(tm, lo, hi), bf16=False)[0][-1]
        fd[j] = np.sum(gc * (fp - fm)) / (2 * h)
    assert rel(gt, fd) < 3e-2
    sur.close()


def _tiny_problem(nside=4, n_steps=64):
    return inputs.config5_problem().replace(nside=nside, n_steps=n_steps)


def test_judge_passes_exact_and_falls_back(torch):
    import paper_2410_01136_gb300 as sx
    sur, _, _, _, sign, rows = small(torch, n_theta=16, nside=4, n_basis=64, map_chunk=3)
    prob = _tiny_problem()
    thetas = inputs.config5_thetas(5, seed=77)
    N = 192
    maps = torch.stack([sx.forward(prob.with_theta(t))[0] for t in thetas])      # [5, 3, N]
    exact = sur.project(maps)
    c = exact.clone()
    d = 2.0 * math.sqrt(N / 64)          # constant offset -> rms 2 K on Q
    c[1, 1, :] += d
    c[3, 2, :] += 0.5 * d                # rms 1 K: not above the threshold... exactly at it
    c[4, 0, :] += 0.4 * d                # rms 0.8 K: kept
    before = c.clone()
    c, rms, fell = sur.judge(prob, thetas, c, rms_max_k=1.0)
    rms = rms.cpu().numpy()
    fell = fell.cpu().numpy()
    ref = so.judge_rms(before.cpu().numpy(), exact.cpu().numpy(), 4)
    assert np.allclose(rms, ref, rtol=1e-4, atol=1e-4)
    assert fell.tolist() == [0, 1, 0, int(rms[3].max() > 1.0), 0]
    assert torch.equal(c[1], exact[1])
    assert torch.equal(c[4], before[4]) and torch.equal(c[0], before[0])
    sur.close()


def test_dataset_normalization_matches_oracle_maps(torch):
    import oracle
    sur, _, _, _, sign, rows = small(torch, n_theta=16, nside=4, n_basis=64, batch=64, map_chunk=40)
    prob = _tiny_problem()
    thetas = inputs.config5_thetas(96, seed=78)
    sur.dataset(prob, thetas)
    mean, scale = sur.normalization()
    lib = oracle.build()
    maps = np.stack([oracle.forward(prob.with_theta(t), threads=4)[0] for t in thetas])     # [n, 3, N]
    c = so.project(maps, 4, sign, rows).reshape(96, -1)
    ref_mean = c.mean(axis=0)
    ref_scale = math.sqrt(np.mean((c - ref_mean) ** 2))
    assert abs(scale - ref_scale) <= 1e-4 * ref_scale
    assert np.max(np.abs(mean - ref_mean)) <= 1e-4 * ref_scale + 1e-5 * np.max(np.abs(ref_mean))
    sur.close()


def test_training_reduces_loss_and_resumes_bitwise(torch, tmp_path):
    def make():
        s, _, _, _, _, _ = small(torch, n_theta=16, nside=4, n_basis=64, batch=64, map_chunk=64,
                                 lr=2e-3, lr_min=1e-4, total_steps=300)
        return s
    prob = _tiny_problem()
    thetas = inputs.config5_thetas(256, seed=79)
    a = make()
    a.dataset(prob, thetas)
    first = a.train(100, seed=5)
    assert np.all(np.isfinite(first))
    a.save(tmp_path / "ck.bin")
    cont_a = a.train(150, seed=5)
    assert cont_a[-20:].mean() < 0.5 * first[:5].mean()
    b = make()
    b.dataset(prob, thetas)
    b.load(tmp_path / "ck.bin")
    cont_b = b.train(150, seed=5)
    assert np.array_equal(cont_a, cont_b)
    for (wa, ba), (wb, bb) in zip(a.params(), b.params()):
        assert np.array_equal(wa, wb) and np.array_equal(ba, bb)
    a.close()
    b.close()


def test_invalid_configurations_are_rejected(torch):
    from paper_2410_01136_gb300 import _native
    from paper_2410_01136_gb300.surrogate import Surrogate
    sign, rows = inputs.surrogate_basis_spec(4, 64, seed=1)
    lo, hi = np.zeros(3), np.ones(3)
    for kw in ({"width": 100}, {"batch": 100}, {"depth": 0}, {"nside": 2}):
        with pytest.raises(_native.SynaxError):
            Surrogate(3, lo, hi, sign, rows, **{"nside": 4, **kw})
    bad = rows.copy()
    bad[1] = bad[0]
    with pytest.raises(_native.SynaxError):
        Surrogate(3, lo, hi, sign, bad, nside=4)
    with pytest.raises(_native.SynaxError):
        Surrogate(3, hi, lo, sign, rows, nside=4)


def test_gate_mean_and_disagreement_match_oracle(torch):
    a, pa, lo, hi, sign, rows = small(torch, seed=1)
    b, pb, _, _, _, _ = small(torch, seed=2)
    mean = np.linspace(-1, 1, a.n_out).astype(np.float32)
    for s_ in (a, b):
        s_.set_normalization(mean, 1.5)
    theta, _ = _batch(torch, a, lo, hi, 15, n=37)
    c, d = a.gate(b, torch.tensor(theta, device="cuda"))
    c = c.cpu().numpy().reshape(37, -1)
    d = d.cpu().numpy()
    x = so.normalize_theta(theta.astype(np.float64), lo, hi)
    ca = mean + 1.5 * so.mlp_forward([(W.astype(np.float64), v.astype(np.float64)) for W, v in pa], x)[0][-1]
    cb = mean + 1.5 * so.mlp_forward([(W.astype(np.float64), v.astype(np.float64)) for W, v in pb], x)[0][-1]
    assert_close(c - mean, 0.5 * (ca + cb) - mean, "gated mean")
    ref = so.judge_rms(ca.reshape(37, 3, -1), cb.reshape(37, 3, -1), 4)
    assert np.allclose(d, ref, rtol=2e-2, atol=1e-3 * ref.max())
    a.close()
    b.close()
