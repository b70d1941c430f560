"""Hamiltonian Monte Carlo over an ensemble of chains on the batch
(synax_hmc_* in include/synax.h): argument marshalling, a warm-up that
adapts the step size and the diagonal mass between runs, and the effective
sample size of the draws.

    hmc = HMC(problems, targets, sigma, theta0, step_size=1e-3, n_leapfrog=8,
              inv_mass=[1, 1, 1, 1, 0, 0, 0, 0])       # 0: parameter held fixed
    hmc.warmup(100)                                    # adapt eps and the mass
    draws, accepted = hmc.run(200)                     # [200, chains, n_theta] on the GPU
    ess = effective_sample_size(draws.cpu().numpy())   # per parameter, all chains

Every step of an iteration (momentum draws, leapfrog updates, the batch
gradients, the Metropolis step) runs in the library's kernels; the warm-up's
adaptation and the effective sample size are host-side statistics of the
draws.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import check, lib


class HMC:
    """HMC chains, one per problem (parameter set) of a batch plan; each
    samples exp(-chi^2/2) against its target times a uniform prior on [lo, hi]."""

    def __init__(self, problems, targets, sigma: float, theta0, step_size: float, n_leapfrog: int, seed: int = 0,
                 inv_mass=None, lo=None, hi=None):
        import torch
        from . import BatchPlan
        self._torch = torch
        self.plan = BatchPlan(problems)
        self.C, self.T = len(problems), len(problems[0].theta)
        th0 = np.ascontiguousarray(np.asarray(theta0, dtype=np.float64).reshape(self.C, self.T))
        self._targets = list(targets)
        keep = []

        def arr(v):
            if v is None:
                return None
            a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(self.T))
            keep.append(a)
            return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

        cfg = _native.SynaxHmcCfg()
        cfg.n_leapfrog, cfg.step_size, cfg.seed = int(n_leapfrog), float(step_size), int(seed) & 0xFFFFFFFFFFFFFFFF
        cfg.inv_mass, cfg.lo, cfg.hi = arr(inv_mass), arr(lo), arr(hi)
        self.inv_mass = np.ones(self.T) if inv_mass is None else np.asarray(inv_mass, dtype=np.float64).copy()
        self.step_size = float(step_size)
        tarr = (ctypes.c_void_p * self.C)(*[t.data_ptr() for t in self._targets])
        h = ctypes.c_void_p()
        check(lib().synax_hmc_create(self.plan._h, ctypes.byref(cfg), th0.ctypes.data_as(ctypes.c_void_p), tarr,
                                     ctypes.c_double(float(sigma)), ctypes.byref(h)), "synax_hmc_create")
        self._h = h

    def _stream(self):
        return ctypes.c_void_p(self._torch.cuda.current_stream().cuda_stream)

    def run(self, n_iters: int, keep_draws: bool = True):
        """n_iters iterations; returns (draws [n_iters, C, T] float64 or None,
        accepted [n_iters, C] int8), CUDA tensors."""
        torch = self._torch
        draws = torch.empty((n_iters, self.C, self.T), dtype=torch.float64, device="cuda") if keep_draws else None
        acc = torch.empty((n_iters, self.C), dtype=torch.int8, device="cuda")
        check(lib().synax_hmc_run(self._h, int(n_iters), ctypes.c_void_p(draws.data_ptr() if draws is not None else 0),
                                  ctypes.c_void_p(acc.data_ptr()), self._stream()), "synax_hmc_run")
        return draws, acc

    def set(self, step_size: float = 0.0, inv_mass=None) -> None:
        ptr = None
        if inv_mass is not None:
            im = np.ascontiguousarray(np.asarray(inv_mass, dtype=np.float64).reshape(self.T))
            self.inv_mass = im.copy()
            ptr = im.ctypes.data_as(ctypes.c_void_p)
        if step_size:
            self.step_size = float(step_size)
        check(lib().synax_hmc_set(self._h, ctypes.c_double(float(step_size)), ptr), "synax_hmc_set")

    def state(self):
        """(theta [C, T], chi2 [C], accepted counts [C]) as CUDA tensors."""
        torch = self._torch
        th = torch.empty((self.C, self.T), dtype=torch.float64, device="cuda")
        c2 = torch.empty(self.C, dtype=torch.float64, device="cuda")
        na = torch.empty(self.C, dtype=torch.int32, device="cuda")
        check(lib().synax_hmc_state(self._h, ctypes.c_void_p(th.data_ptr()), ctypes.c_void_p(c2.data_ptr()),
                                    ctypes.c_void_p(na.data_ptr()), self._stream()), "synax_hmc_state")
        return th, c2, na

    def warmup(self, n_iters: int, target_accept: float = 0.7, window: int = 5, adapt_mass: bool = True) -> list:
        """Runs n_iters iterations in windows of `window`.  After each window
        the step size is scaled by exp(3 (acceptance - target)).  Halfway, the
        free parameters' inverse masses become the variance of the draws of
        the second quarter (after the start-up transient), a diagonal
        estimate of the posterior covariance, and the step size is rescaled
        so that the typical position step eps sqrt(inv_mass) is unchanged
        (geometric mean over the free parameters); adapt_mass=False keeps the
        given mass (e.g. a Laplace estimate).  Returns the (step size,
        acceptance) history."""
        hist = []
        free = self.inv_mass > 0
        done, mass_set, seen = 0, not adapt_mass, []
        while done < n_iters:
            k = min(window, n_iters - done)
            draws, acc = self.run(k)
            seen.append((done, draws))
            a = float(acc.float().mean().item())
            hist.append((self.step_size, a))
            done += k
            eps = self.step_size * float(np.exp(3.0 * (a - target_accept)))
            if not mass_set and done >= n_iters // 2:
                mass_set = True
                part = [d for start, d in seen if start >= n_iters // 4] or [d for _, d in seen]
                var = self._torch.cat(part).reshape(-1, self.T).var(dim=0).cpu().numpy()
                if np.all(var[free] > 0):
                    ratio = float(np.exp(np.mean(np.log(self.inv_mass[free] / var[free]))))
                    self.set(eps * np.sqrt(ratio), np.where(free, var, 0.0))
                    continue
            self.set(eps)
        return hist

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().synax_hmc_destroy(self._h)
            self._h = None
        if getattr(self, "plan", None) is not None:
            self.plan.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def laplace_inv_mass(prob, target, sigma: float, free, h_rel: float = 1e-3) -> np.ndarray:
    """Diagonal Laplace estimate of the posterior variance of the free
    parameters at prob.theta: U = chi^2 / 2 has curvature U''_jj =
    (g_j(theta + h e_j) - g_j(theta - h e_j)) / (4 h) with g = d chi^2 / d theta
    from synax_adjoint; the variance is 1 / U''_jj (0 for fixed parameters,
    and where the curvature is not positive)."""
    from . import adjoint
    th = np.asarray(prob.theta, dtype=np.float64)
    out = np.zeros(th.size)
    for j in free:
        h = h_rel * max(abs(th[j]), 1e-3)
        e = np.zeros(th.size)
        e[j] = h
        gp, _ = adjoint(prob.with_theta(th + e), target=target, sigma=sigma)
        gm, _ = adjoint(prob.with_theta(th - e), target=target, sigma=sigma)
        curv = (float(gp[j].item()) - float(gm[j].item())) / (4.0 * h)
        out[j] = 1.0 / curv if curv > 0 else 0.0
    return out


def effective_sample_size(draws) -> np.ndarray:
    """Multi-chain effective sample size per parameter of draws [n, m, k]
    (n draws, m chains), after Gelman et al., Bayesian Data Analysis (3rd
    ed.), Sec. 11.5: rho_t = 1 - (W - mean autocovariance_t) / var+, summed
    over Geyer's initial positive and monotone sequence of pair sums;
    ESS = m n / (-1 + 2 sum of the pair sums), capped at m n log10(m n) (as
    Stan does); 0 for chains that do not move (no within-chain variance)."""
    x = np.asarray(draws, dtype=np.float64)
    n, m, k = x.shape
    out = np.empty(k)
    for j in range(k):
        y = x[:, :, j] - x[:, :, j].mean(axis=0, keepdims=True)
        f = np.fft.rfft(y, n=2 * n, axis=0)
        acov = np.fft.irfft(f * np.conj(f), axis=0)[:n] / n          # biased autocovariance per chain
        W = acov[0].mean() * n / (n - 1)
        B_over_n = x[:, :, j].mean(axis=0).var(ddof=1) if m > 1 else 0.0
        var_plus = W * (n - 1) / n + B_over_n
        scale = max(float(np.abs(x[:, :, j]).max()), 1e-300)
        if not W > (1e-14 * scale) ** 2:
            out[j] = 0.0
            continue
        rho = 1.0 - (W - acov.mean(axis=1)) / var_plus
        rho[0] = 1.0
        tau, prev = -1.0, np.inf
        for t in range(0, n - 1, 2):
            pair = rho[t] + rho[t + 1]
            if pair <= 0:
                break
            pair = min(pair, prev)
            tau += 2.0 * pair
            prev = pair
        out[j] = min(m * n / max(tau, 1e-12), m * n * np.log10(m * n))
    return out
