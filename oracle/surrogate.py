"""FP64 oracle of the learned surrogate -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may import this module; the product never does, and this module
imports nothing of the product.  Plain numpy in double precision, written
for checking by eye:

* the basis the surrogate's outputs are coordinates in: a subsampled
  randomized Hadamard transform (Ailon & Chazelle 2006) of a HEALPix map,
  e_i[p] = s_p H_N[r_i, p] / sqrt(N), N = 12 Nside^2, with seeded signs s_p
  and seeded distinct rows r_i, and H_N = H_12 (x) H_M (M = Nside^2) the
  Kronecker product of the Paley Hadamard matrix of order 12 and the
  Sylvester one of order M.  Its rows are orthonormal, so a coefficient
  residual measures the map residual inside the spanned subspace;
* the projection c_i = sum_p e_i[p] m_p of a map, and the judge's RMS
  ||c - c'||_2 / sqrt(N) per Stokes parameter;
* the multilayer perceptron (widths 16 -> 1024 x 4 with GELU -> 9216), its
  mean-squared-error loss, the gradients by backpropagation and one Adam step
  (Kingma & Ba 2015, Algorithm 1).  With bf16=True the values that the GPU
  kernels hand to the tensor cores as BF16 operands are rounded to BF16
  (round to nearest even) at the same points; every sum is still FP64.

Parity pins (tests/test_oracle_surrogate.py): H_12 H_12^T = 12 I; the
Sylvester factor against scipy.linalg.hadamard; H_N against numpy.kron;
orthonormality and Parseval by brute force at Nside 1 and 2; GELU's odd
identity and values of the normal CDF; backpropagation against central
finite differences of the loss; Adam's first step in closed form; the BF16
rounding against torch's conversion and hand-worked ties.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf, lpmv

# ---------------------------------------------------------------------------
# basis
# ---------------------------------------------------------------------------


def paley_hadamard12() -> np.ndarray:
    """Hadamard matrix of order 12 by Paley's first construction over GF(11)
    (11 = 3 mod 4): H = I + [[0, 1^T], [-1, Q]], Q_ij = chi(j - i), chi the
    quadratic character mod 11."""
    q = 11
    residues = {(x * x) % q for x in range(1, q)}
    chi = np.array([0] + [1 if a in residues else -1 for a in range(1, q)], dtype=np.int64)
    Q = np.empty((q, q), dtype=np.int64)
    for i in range(q):
        for j in range(q):
            Q[i, j] = chi[(j - i) % q]
    S = np.zeros((q + 1, q + 1), dtype=np.int64)
    S[0, 1:] = 1
    S[1:, 0] = -1
    S[1:, 1:] = Q
    return np.eye(q + 1, dtype=np.int64) + S


def hadamard_entries(rows, cols, nside: int) -> np.ndarray:
    """H_N[rows[:, None], cols[None, :]] with H_N = H_12 (x) H_M, M = nside^2,
    Sylvester H_M[a, b] = (-1)^popcount(a & b)."""
    M = nside * nside
    H12 = paley_hadamard12()
    r = np.asarray(rows, dtype=np.int64)[:, None]
    c = np.asarray(cols, dtype=np.int64)[None, :]
    outer = H12[r // M, c // M]
    a = (r % M) & (c % M)
    parity = np.zeros(a.shape, dtype=np.int64)
    while np.any(a):
        parity ^= a & 1
        a = a >> 1
    return outer * (1 - 2 * parity)


def basis(nside: int, signs, rows) -> np.ndarray:
    """The basis vectors as a dense [K, N] FP64 matrix (rows orthonormal)."""
    N = 12 * nside * nside
    H = hadamard_entries(rows, np.arange(N), nside).astype(np.float64)
    return H * np.asarray(signs, dtype=np.float64)[None, :] / math.sqrt(N)


def project(maps, nside: int, signs, rows, chunk: int = 256) -> np.ndarray:
    """Coefficients c[..., i] = sum_p e_i[p] m[..., p] of maps [..., N]."""
    maps = np.asarray(maps, dtype=np.float64)
    rows = np.asarray(rows)
    out = np.empty(maps.shape[:-1] + (rows.size,), dtype=np.float64)
    for k0 in range(0, rows.size, chunk):
        E = basis(nside, signs, rows[k0:k0 + chunk])
        out[..., k0:k0 + chunk] = maps @ E.T
    return out


def sh_index(l: int, m: int) -> int:
    """Position of the real harmonic (l, m), m in [-l, l], in the basis order."""
    return l * l + l + m


def real_sph_harm_pixels(nside: int, n_basis: int) -> np.ndarray:
    """Real spherical harmonics at the RING pixel centres, [n_basis][npix]:
    Y_l0 = N_l0 P_l^0(cos t), Y_lm = sqrt(2) N_lm P_l^m(cos t) cos(m phi) and
    Y_l,-m = sqrt(2) N_lm P_l^m(cos t) sin(m phi) for m > 0, with
    N_lm = sqrt((2l + 1) / (4 pi) (l - m)! / (l + m)!) and P_l^m the associated
    Legendre function with the Condon-Shortley phase (scipy's lpmv), in the
    order (l, m) -> l^2 + l + m."""
    import oracle
    npix = 12 * nside * nside
    zs = np.empty(npix)
    ph = np.empty(npix)
    for p in range(npix):
        zs[p], ph[p] = oracle.healpix_centre(nside, p)
    out = np.empty((n_basis, npix))
    l = 0
    while l * l < n_basis:
        for m in range(0, l + 1):
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            P = norm * lpmv(m, l, zs)
            if m == 0:
                if sh_index(l, 0) < n_basis:
                    out[sh_index(l, 0)] = P
            else:
                if sh_index(l, m) < n_basis:
                    out[sh_index(l, m)] = math.sqrt(2.0) * P * np.cos(m * ph)
                if sh_index(l, -m) < n_basis:
                    out[sh_index(l, -m)] = math.sqrt(2.0) * P * np.sin(m * ph)
        l += 1
    return out


def cholesky_qr2(Y) -> np.ndarray:
    """Orthonormal rows spanning, for every k, the span of Y's first k rows:
    E = L^-1 Y with G = Y Y^T = L L^T (Cholesky), applied twice."""
    E = np.asarray(Y, dtype=np.float64)
    for _ in range(2):
        L = np.linalg.cholesky(E @ E.T)
        E = np.linalg.solve(L, E)
    return E


def sh_basis(nside: int, n_basis: int) -> np.ndarray:
    """The low-order surrogate basis: real spherical harmonics at the pixel
    centres, orthonormalised in their (l, m) order (cholesky_qr2)."""
    return cholesky_qr2(real_sph_harm_pixels(nside, n_basis))


def judge_rms(c_sur, c_true, nside: int) -> np.ndarray:
    """In-subspace RMS residual per (map, Stokes): ||c_sur - c_true||_2 / sqrt(N)
    over the basis index, for coefficients shaped [..., 3, K]."""
    N = 12 * nside * nside
    d = np.asarray(c_sur, dtype=np.float64) - np.asarray(c_true, dtype=np.float64)
    return np.sqrt(np.sum(d * d, axis=-1) / N)


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------


def bf16_round(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), via FP32; returned as FP64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def gelu(z) -> np.ndarray:
    """GELU(z) = z Phi(z) with the exact normal CDF Phi(z) = (1 + erf(z/sqrt 2))/2."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z) -> np.ndarray:
    """d GELU / dz = Phi(z) + z phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def normalize_theta(theta, lo, hi) -> np.ndarray:
    """Map the training box [lo, hi] onto [-1, 1] per parameter."""
    theta = np.asarray(theta, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return (theta - lo) * (2.0 / (hi - lo)) - 1.0


def _q(x, bf16: bool) -> np.ndarray:
    return bf16_round(x) if bf16 else np.asarray(x, dtype=np.float64)


def mlp_forward(params, x, bf16: bool = True):
    """Forward pass.  params: [(W [out, in], b [out])]; x [B, in].
    Returns (zs, xs): zs[l] the pre-activation of layer l, xs[l] the operand
    that layer l multiplies (xs[0] the input); the last z is the output."""
    xs = [_q(x, bf16)]
    zs = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = xs[-1] @ _q(W, bf16).T + np.asarray(b, dtype=np.float64)[None, :]
        zs.append(z)
        if l < L - 1:
            xs.append(_q(gelu(z), bf16))
    return zs, xs


def mlp_backward(params, zs, xs, dout, bf16: bool = True):
    """Backpropagate dL/d(output) `dout` [B, n_out] (already in the operand
    precision).  Returns ([(dW, db)], dL/dx of the network input)."""
    L = len(params)
    grads = [None] * L
    d = np.asarray(dout, dtype=np.float64)
    dx = None
    for l in range(L - 1, -1, -1):
        W = _q(params[l][0], bf16)
        grads[l] = (d.T @ xs[l], d.sum(axis=0))
        back = d @ W
        if l > 0:
            d = _q(back * gelu_grad(zs[l - 1]), bf16)
        else:
            dx = back
    return grads, dx


def mse_loss_and_grads(params, x, y, bf16: bool = True):
    """L = mean over batch and outputs of (f(x) - y)^2, and its gradients."""
    zs, xs = mlp_forward(params, x, bf16)
    out = zs[-1]
    diff = out - np.asarray(y, dtype=np.float64)
    loss = float(np.mean(diff * diff))
    dout = _q(2.0 * diff / diff.size, bf16)
    grads, _ = mlp_backward(params, zs, xs, dout, bf16)
    return loss, grads


def adam_step(w, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update at step t >= 1 (bias-corrected moments).  Returns (w, m, v)."""
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def cosine_lr(t: int, lr0: float, lr_min: float, total: int) -> float:
    """Learning rate at step t: cosine decay from lr0 to lr_min over `total` steps."""
    s = min(t, total) / max(total, 1)
    return lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * s))
