"""Pins of the surrogate oracle against closed forms, library routines and
brute force (no GPU)."""
import math

import numpy as np
import pytest

from oracle import surrogate as so
from paper_2410_01136_gb300 import inputs


def test_paley_order12_is_hadamard():
    H = so.paley_hadamard12()
    assert set(np.unique(H)) == {-1, 1}
    assert np.array_equal(H @ H.T, 12 * np.eye(12, dtype=np.int64))


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_hadamard_is_kronecker_of_paley_and_sylvester(nside):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    M = nside * nside
    N = 12 * M
    H = so.hadamard_entries(np.arange(N), np.arange(N), nside)
    ref = np.kron(so.paley_hadamard12(), scipy_linalg.hadamard(M))
    assert np.array_equal(H, ref)
    assert np.array_equal(H @ H.T, N * np.eye(N, dtype=np.int64))


@pytest.mark.parametrize("nside", [1, 2])
def test_full_basis_is_orthonormal_and_parseval(nside):
    N = 12 * nside * nside
    signs, rows = inputs.surrogate_basis_spec(nside, N, seed=5)
    assert sorted(rows.tolist()) == list(range(N))
    E = so.basis(nside, signs, rows)
    assert np.allclose(E @ E.T, np.eye(N), atol=1e-13)
    assert np.allclose(E.T @ E, np.eye(N), atol=1e-13)
    m = np.random.default_rng(0).normal(size=(3, N))
    c = so.project(m, nside, signs, rows)
    assert np.allclose(np.linalg.norm(c, axis=-1), np.linalg.norm(m, axis=-1), rtol=1e-13)
    # brute force: each coefficient is the plain dot product with its vector
    for i in range(0, N, 7):
        e = np.array([signs[p] * (1 if _brute_h(rows[i], p, nside) > 0 else -1) for p in range(N)]) / math.sqrt(N)
        assert abs(c[1, i] - e @ m[1]) < 1e-12


def _brute_h(r, c, nside):
    """H_N[r, c] from the Kronecker definition, one bit at a time."""
    M = nside * nside
    h = so.paley_hadamard12()[r // M, c // M]
    a, b = r % M, c % M
    while a or b:
        if (a & 1) and (b & 1):
            h = -h
        a >>= 1
        b >>= 1
    return h


def test_subset_basis_residual_is_in_subspace_norm():
    nside = 2
    N = 48
    signs, rows = inputs.surrogate_basis_spec(nside, 12, seed=9)
    E = so.basis(nside, signs, rows)
    assert np.allclose(E @ E.T, np.eye(12), atol=1e-13)
    rng = np.random.default_rng(1)
    m1, m2 = rng.normal(size=(2, 3, N))
    c1, c2 = so.project(m1, nside, signs, rows), so.project(m2, nside, signs, rows)
    # residual of coefficients == RMS of the projected map residual
    proj = (c1 - c2) @ E
    assert np.allclose(so.judge_rms(c1, c2, nside), np.sqrt(np.sum(proj ** 2, axis=-1) / N), rtol=1e-12)


def test_basis_spec_is_seeded_and_distinct():
    s1, r1 = inputs.surrogate_basis_spec(64, 3072, seed=5)
    s2, r2 = inputs.surrogate_basis_spec(64, 3072, seed=5)
    assert np.array_equal(s1, s2) and np.array_equal(r1, r2)
    assert len(set(r1.tolist())) == 3072 and r1.min() >= 0 and r1.max() < 49152
    assert abs(float(np.mean(s1))) < 0.02


def test_bf16_rounding_ties_and_torch():
    torch = pytest.importorskip("torch")
    one = 1.0
    ulp = 2.0 ** -7
    assert so.bf16_round(one + ulp / 2) == one                # tie -> even (1.0)
    assert so.bf16_round(one + 3 * ulp / 2) == one + 2 * ulp  # tie -> even (odd mantissa rounds up)
    assert so.bf16_round(one + ulp / 2 + 2.0 ** -20) == one + ulp
    assert so.bf16_round(-3.0) == -3.0
    x = np.random.default_rng(2).normal(size=4096) * np.exp(np.random.default_rng(3).normal(size=4096) * 5)
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).float().double().numpy()
    assert np.array_equal(so.bf16_round(x), ref)


def test_gelu_identities():
    z = np.linspace(-6, 6, 97)
    assert np.allclose(so.gelu(z) - so.gelu(-z), z, atol=1e-15)       # z Phi(z) + z Phi(-z) = z
    assert so.gelu(0.0) == 0.0
    assert abs(so.gelu(1.0) - 0.8413447460685429) < 1e-15              # Phi(1) (standard normal table)
    assert abs(so.gelu(-1.959963984540054) + 1.959963984540054 * 0.025) < 1e-13
    h = 1e-6
    fd = (so.gelu(z + h) - so.gelu(z - h)) / (2 * h)
    assert np.allclose(so.gelu_grad(z), fd, atol=1e-9)


def _small_params(seed=0, widths=(5, 7, 6, 4)):
    rng = np.random.default_rng(seed)
    return [(rng.normal(size=(widths[l + 1], widths[l])) / math.sqrt(widths[l]),
             rng.normal(size=widths[l + 1]) * 0.1) for l in range(len(widths) - 1)]


def test_backprop_matches_central_differences():
    params = _small_params()
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, size=(9, 5))
    y = rng.normal(size=(9, 4))
    loss, grads = so.mse_loss_and_grads(params, x, y, bf16=False)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2)]:
            Wp = [(w.copy(), bb.copy()) for w, bb in params]
            Wm = [(w.copy(), bb.copy()) for w, bb in params]
            Wp[l][0][i, j] += h
            Wm[l][0][i, j] -= h
            fd = (so.mse_loss_and_grads(Wp, x, y, False)[0] - so.mse_loss_and_grads(Wm, x, y, False)[0]) / (2 * h)
            assert abs(grads[l][0][i, j] - fd) < 1e-7 * max(1.0, abs(fd))
        for i in range(b.size):
            Bp = [(w.copy(), bb.copy()) for w, bb in params]
            Bm = [(w.copy(), bb.copy()) for w, bb in params]
            Bp[l][1][i] += h
            Bm[l][1][i] -= h
            fd = (so.mse_loss_and_grads(Bp, x, y, False)[0] - so.mse_loss_and_grads(Bm, x, y, False)[0]) / (2 * h)
            assert abs(grads[l][1][i] - fd) < 1e-7 * max(1.0, abs(fd))


def test_input_gradient_matches_central_differences():
    params = _small_params(3)
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, size=(4, 5))
    g = rng.normal(size=(4, 4))
    zs, xs = so.mlp_forward(params, x, bf16=False)
    _, dx = so.mlp_backward(params, zs, xs, g, bf16=False)
    h = 1e-6
    for i in range(5):
        e = np.zeros(5)
        e[i] = h
        fp = np.sum(so.mlp_forward(params, x + e, False)[0][-1] * g, axis=1)
        fm = np.sum(so.mlp_forward(params, x - e, False)[0][-1] * g, axis=1)
        assert np.allclose(dx[:, i], (fp - fm) / (2 * h), atol=1e-7)


def test_adam_first_step_closed_form():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    w0 = np.array([1.0, 2.0, 3.0, 4.0])
    w, m, v = so.adam_step(w0, g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-8)
    # bias-corrected first moments are g and g^2: the step is lr * g / (|g| + eps)
    assert np.allclose(w, w0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_cosine_lr_endpoints():
    assert so.cosine_lr(0, 1e-3, 1e-5, 100) == 1e-3
    assert abs(so.cosine_lr(100, 1e-3, 1e-5, 100) - 1e-5) < 1e-18
    assert abs(so.cosine_lr(50, 1e-3, 1e-5, 100) - 0.5 * (1e-3 + 1e-5)) < 1e-15
    assert so.cosine_lr(500, 1e-3, 1e-5, 100) == so.cosine_lr(100, 1e-3, 1e-5, 100)


# ---------------------------------------------------------------------------
# low-order basis: real spherical harmonics at the pixel centres
# ---------------------------------------------------------------------------

def test_sh_values_match_scipy():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    import oracle
    from oracle import surrogate as osur
    nside, nb = 4, 49                                   # l <= 6
    Y = osur.real_sph_harm_pixels(nside, nb)
    for p in (0, 7, 50, 95, 140, 191):
        z, phi = oracle.healpix_centre(nside, p)
        t = np.arccos(z)
        for l in range(7):
            for m in range(-l, l + 1):
                c = sp.sph_harm_y(l, abs(m), t, phi)      # complex, Condon-Shortley phase
                want = c.real if m == 0 else np.sqrt(2.0) * (c.real if m > 0 else c.imag)
                assert Y[osur.sh_index(l, m), p] == pytest.approx(want, abs=1e-12)


def test_sh_basis_orthonormal_and_nested():
    from oracle import surrogate as osur
    nside, nb = 4, 64
    Y = osur.real_sph_harm_pixels(nside, nb)
    E = osur.sh_basis(nside, nb)
    np.testing.assert_allclose(E @ E.T, np.eye(nb), atol=1e-12)
    # nested: the first k rows of E span the first k harmonics (E = L^-1 Y, lower triangular)
    for k in (1, 4, 9, 16, 36):
        R = Y[:k] @ E[:k].T                              # coordinates of Y_i in the first k rows of E
        np.testing.assert_allclose(R @ E[:k], Y[:k], atol=1e-11)
    # the monopole: a constant map has only its first coefficient
    c = E @ np.ones(12 * nside * nside)
    assert abs(c[0]) == pytest.approx(np.sqrt(12 * nside * nside), rel=1e-12)
    np.testing.assert_allclose(c[1:], 0.0, atol=1e-11)
