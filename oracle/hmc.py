"""Plain HMC and the effective sample size, for checking the library's
sampler -- TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

hmc_chain follows the algorithm of Neal, "MCMC using Hamiltonian dynamics"
(Handbook of MCMC, 2011), Sec. 5.2-5.3: momentum p ~ N(0, M) with diagonal
M = diag(1 / inv_mass) (a zero inverse mass holds a parameter fixed), L
leapfrog steps of size eps for U = chi^2 / 2 (a half step of the momentum, L
full position steps with L - 1 full momentum steps between them, a final
half step), and a Metropolis step on H = U + p^T M^-1 p / 2, rejecting
proposals outside the prior box.  The random numbers are those the library
documents (include/synax.h, synax_hmc_*), drawn with the seeded SplitMix64
stream of paper_2410_01136_gb300.inputs.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2410_01136_gb300 import inputs

ACCEPT_STREAM = 0x632BE59BD9B4E019


def momentum_normals(seed: int, t: int, C: int, T: int) -> np.ndarray:
    """z [C, T]: pair k = (t C + c) T + j of stream `seed`, first Box-Muller output."""
    k0 = t * C * T
    raw = inputs.splitmix64(seed, 2 * C * T, offset=2 * k0)
    u1 = ((raw[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (raw[1::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)).reshape(C, T)


def accept_uniforms(seed: int, t: int, C: int) -> np.ndarray:
    raw = inputs.splitmix64((seed + ACCEPT_STREAM) & 0xFFFFFFFFFFFFFFFF, C, offset=t * C)
    return (raw >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def hmc_iterations(theta, chi2_and_grad, n_iters: int, eps: float, L: int, seed: int, inv_mass, lo=None, hi=None,
                   t0: int = 0):
    """Runs n_iters HMC iterations for C chains at once (theta [C, T]);
    chi2_and_grad(theta [C, T]) -> (chi2 [C], d chi^2 / d theta [C, T]).
    Returns (draws [n_iters, C, T], accepted [n_iters, C])."""
    theta = np.array(theta, dtype=np.float64)
    C, T = theta.shape
    im = np.asarray(inv_mass, dtype=np.float64)
    lo = np.full(T, -np.inf) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.full(T, np.inf) if hi is None else np.asarray(hi, dtype=np.float64)
    chi2, g = chi2_and_grad(theta)
    draws = np.empty((n_iters, C, T))
    accepted = np.empty((n_iters, C), dtype=np.int8)
    for it in range(n_iters):
        t = t0 + it
        z = momentum_normals(seed, t, C, T)
        p = np.where(im > 0, z / np.sqrt(np.where(im > 0, im, 1.0)), 0.0)
        H0 = 0.5 * chi2 + 0.5 * np.sum(im * p * p, axis=1)
        th = theta.copy()
        p = p - 0.5 * eps * 0.5 * g
        th = th + eps * im * p
        for l in range(1, L + 1):
            c2, gl = chi2_and_grad(th)
            if l < L:
                p = p - eps * 0.5 * gl
                th = th + eps * im * p
            else:
                p = p - 0.5 * eps * 0.5 * gl
        H1 = 0.5 * c2 + 0.5 * np.sum(im * p * p, axis=1)
        u = accept_uniforms(seed, t, C)
        inside = np.all((th >= lo) & (th <= hi), axis=1)
        with np.errstate(divide="ignore", invalid="ignore"):
            ok = inside & np.isfinite(H1) & ((u == 0.0) | (np.log(u) < H0 - H1))
        theta = np.where(ok[:, None], th, theta)
        chi2 = np.where(ok, c2, chi2)
        g = np.where(ok[:, None], gl, g)
        draws[it] = theta
        accepted[it] = ok
    return draws, accepted
