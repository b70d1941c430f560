"""Python binding of the learned surrogate (synax_surrogate_* in include/synax.h).

Argument marshalling only: every step (basis, projection, training maps,
forward/backward passes, Adam, judging) runs in the CUDA library.

    sur = Surrogate.for_workload()                       # 16 -> 1024 x 4 -> 3 x 3072
    sur.dataset(problem, thetas)                         # render + project training maps
    losses = sur.train(n_steps, seed)                    # graph-captured Adam steps
    c = sur(theta)                                       # [n, 3, n_basis] coefficients
    c, g = sur(theta, gcoeff)                            # and dL/dtheta for seed dL/dc
    c, rms, fell = sur.judge(problem, thetas, c, 1.0)    # march-judged, with fallback
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native, inputs
from ._native import check, lib


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _stream(torch):
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Surrogate:
    """A surrogate handle.  theta_lo/theta_hi: the input box (physical units);
    basis_sign/basis_rows: the basis draws (inputs.surrogate_basis_spec);
    init: the initial flat parameters or a list of (W, b) (inputs.mlp_init)."""

    def __init__(self, n_theta, theta_lo, theta_hi, basis_sign, basis_rows, *, width=1024, depth=4, nside=64,
                 batch=512, max_eval=16384, map_chunk=128, total_steps=10000, lr=1e-3, lr_min=1e-5,
                 beta1=0.9, beta2=0.999, eps=1e-8, init=None, basis="srht", n_basis=None):
        import torch
        self._torch = torch
        cfg = _native.SynaxSurrogateCfg()
        cfg.n_theta, cfg.width, cfg.depth, cfg.nside = n_theta, width, depth, nside
        if basis not in ("srht", "sh"):
            raise ValueError("basis is 'srht' (seeded +-1 rows) or 'sh' (spherical harmonics)")
        self.basis = basis
        cfg.basis_kind = _native.SUR_BASIS_SRHT if basis == "srht" else _native.SUR_BASIS_SH
        self.n_basis = int(len(basis_rows)) if basis == "srht" else int(n_basis)
        cfg.n_basis, cfg.batch, cfg.max_eval, cfg.map_chunk = self.n_basis, batch, max_eval, map_chunk
        cfg.total_steps, cfg.lr, cfg.lr_min = total_steps, lr, lr_min
        cfg.beta1, cfg.beta2, cfg.eps = beta1, beta2, eps
        lo = np.asarray(theta_lo, dtype=np.float64)
        hi = np.asarray(theta_hi, dtype=np.float64)
        for j in range(n_theta):
            cfg.theta_lo[j] = float(lo[j])
            cfg.theta_hi[j] = float(hi[j])
        if basis == "srht":
            self._sign = np.ascontiguousarray(basis_sign, dtype=np.int8)
            self._rows = np.ascontiguousarray(basis_rows, dtype=np.int32)
            cfg.basis_sign = self._sign.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
            cfg.basis_rows = self._rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        h = ctypes.c_void_p()
        check(lib().synax_surrogate_create(ctypes.byref(cfg), ctypes.byref(h)), "synax_surrogate_create")
        self._h = h
        self.n_theta, self.width, self.depth, self.nside, self.batch = n_theta, width, depth, nside, batch
        self.npix = 12 * nside * nside
        self.n_out = 3 * self.n_basis
        self.theta_lo, self.theta_hi = lo[:n_theta].copy(), hi[:n_theta].copy()
        self.widths = (n_theta,) + (width,) * depth + (self.n_out,)
        if init is not None:
            self.set_params(init)

    @classmethod
    def for_workload(cls, **kw):
        """The Nside-64 JF12-type surrogate: 16 -> 1024 x 4 -> 3 x 3072, box
        theta_fid -/+ 20 % of each parameter's scale, init seed 7; basis
        'srht' (seed 5) or 'sh' (the first 3072 real harmonics, l <= 55)."""
        lo, hi = inputs.config5_box()
        init_seed = kw.pop("init_seed", 7)
        if kw.get("basis", "srht") == "sh":
            kw.pop("basis_seed", None)
            sur = cls(16, lo, hi, None, None, n_basis=3072, **kw)
        else:
            sign, rows = inputs.surrogate_basis_spec(64, 3072, seed=kw.pop("basis_seed", 5))
            sur = cls(16, lo, hi, sign, rows, **kw)
        sur.set_params(inputs.mlp_init(sur.widths, seed=init_seed))
        return sur

    # ---- parameters and state ----
    @property
    def n_params(self) -> int:
        return int(lib().synax_surrogate_param_count(self._h))

    def _flat(self, layers) -> np.ndarray:
        parts = []
        for W, b in layers:
            parts += [np.asarray(W, dtype=np.float32).ravel(), np.asarray(b, dtype=np.float32).ravel()]
        return np.concatenate(parts)

    def _layers(self, flat) -> list:
        out, o = [], 0
        for l in range(len(self.widths) - 1):
            k, n = self.widths[l], self.widths[l + 1]
            W = flat[o:o + n * k].reshape(n, k)
            o += n * k
            b = flat[o:o + n]
            o += n
            out.append((W, b))
        return out

    def set_params(self, params) -> None:
        flat = params if isinstance(params, np.ndarray) and params.ndim == 1 else self._flat(params)
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        check(lib().synax_surrogate_set_params(self._h, flat.ctypes.data_as(ctypes.c_void_p), flat.size),
              "synax_surrogate_set_params")

    def _get(self, what: int, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.float32)
        check(lib().synax_surrogate_get(self._h, what, out.ctypes.data_as(ctypes.c_void_p), n), "synax_surrogate_get")
        return out

    def params(self) -> list:
        return self._layers(self._get(_native.SUR_PARAMS, self.n_params))

    def grads(self) -> list:
        return self._layers(self._get(_native.SUR_GRADS, self.n_params))

    def adam_moments(self) -> tuple[list, list]:
        return (self._layers(self._get(_native.SUR_ADAM_M, self.n_params)),
                self._layers(self._get(_native.SUR_ADAM_V, self.n_params)))

    def normalization(self) -> tuple[np.ndarray, float]:
        v = self._get(_native.SUR_NORM, self.n_out + 1)
        return v[:-1].copy(), float(v[-1])

    def set_normalization(self, mean, scale: float) -> None:
        m = np.ascontiguousarray(mean, dtype=np.float32)
        check(lib().synax_surrogate_set_normalization(self._h, m.ctypes.data_as(ctypes.c_void_p), float(scale)),
              "synax_surrogate_set_normalization")

    def losses(self, n: int) -> np.ndarray:
        return self._get(_native.SUR_LOSS, n)

    # ---- basis ----
    def project(self, maps):
        """maps [..., npix] (device float32) -> coefficients [..., n_basis]."""
        torch = self._torch
        m = maps.contiguous()
        rows = m.numel() // self.npix
        out = torch.empty(m.shape[:-1] + (self.n_basis,), dtype=torch.float32, device=m.device)
        check(lib().synax_surrogate_project(self._h, _ptr(m), rows, _ptr(out), _stream(torch)),
              "synax_surrogate_project")
        return out

    # ---- training ----
    def dataset(self, prob, thetas) -> None:
        th = np.ascontiguousarray(thetas, dtype=np.float64)
        ps = _native.problem_struct(prob)
        check(lib().synax_surrogate_dataset(self._h, ctypes.byref(ps), th.ctypes.data_as(ctypes.c_void_p),
                                            th.shape[0], _stream(self._torch)), "synax_surrogate_dataset")

    def step(self, theta, coeffs, update: bool = True):
        """One pass on an explicit batch (device tensors); returns the loss (device scalar)."""
        torch = self._torch
        loss = torch.empty(1, dtype=torch.float32, device=theta.device)
        check(lib().synax_surrogate_step(self._h, _ptr(theta.contiguous()), _ptr(coeffs.contiguous()),
                                         theta.shape[0], int(update), _ptr(loss), _stream(torch)),
              "synax_surrogate_step")
        return loss

    def train(self, n_steps: int, seed: int = 0) -> np.ndarray:
        check(lib().synax_surrogate_train(self._h, int(n_steps), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                          _stream(self._torch)), "synax_surrogate_train")
        self.status()
        return self.losses(n_steps) if n_steps else np.empty(0, dtype=np.float32)

    # ---- inference ----
    def __call__(self, theta, gcoeff=None):
        torch = self._torch
        th = theta.contiguous().float()
        n = th.shape[0]
        c = torch.empty((n, 3, self.n_basis), dtype=torch.float32, device=th.device)
        if gcoeff is None:
            check(lib().synax_surrogate(self._h, _ptr(th), n, _ptr(c), None, None, _stream(torch)), "synax_surrogate")
            return c
        g = gcoeff.contiguous().float()
        gt = torch.empty((n, self.n_theta), dtype=torch.float32, device=th.device)
        check(lib().synax_surrogate(self._h, _ptr(th), n, _ptr(c), _ptr(g), _ptr(gt), _stream(torch)),
              "synax_surrogate")
        return c, gt

    def judge(self, prob, thetas, coeffs, rms_max_k: float = 1.0):
        """Judge coefficients (device [n, 3, n_basis], replaced in place where
        the surrogate misses) against the march.  Returns (coeffs, rms [n, 3], fell_back [n])."""
        torch = self._torch
        th = np.ascontiguousarray(thetas, dtype=np.float64)
        n = th.shape[0]
        rms = torch.empty((n, 3), dtype=torch.float32, device=coeffs.device)
        fell = torch.empty(n, dtype=torch.int32, device=coeffs.device)
        ps = _native.problem_struct(prob)
        check(lib().synax_surrogate_judge(self._h, ctypes.byref(ps), th.ctypes.data_as(ctypes.c_void_p), n,
                                          _ptr(coeffs), float(rms_max_k), _ptr(rms), _ptr(fell), _stream(torch)),
              "synax_surrogate_judge")
        return coeffs, rms, fell

    def gate(self, other: "Surrogate", theta):
        """Mean coefficients of this surrogate and `other` and their
        disagreement [n, 3] (in-subspace RMS of the difference, kelvin)."""
        torch = self._torch
        th = theta.contiguous().float()
        n = th.shape[0]
        c = torch.empty((n, 3, self.n_basis), dtype=torch.float32, device=th.device)
        scratch = torch.empty_like(c)
        d = torch.empty((n, 3), dtype=torch.float32, device=th.device)
        check(lib().synax_surrogate_gate(self._h, other._h, _ptr(th), n, _ptr(c), _ptr(scratch), _ptr(d),
                                         _stream(torch)), "synax_surrogate_gate")
        return c, d

    def status(self) -> None:
        check(lib().synax_surrogate_status(self._h, _stream(self._torch)), "synax_surrogate_status")

    # ---- checkpoints ----
    def save(self, path: str) -> None:
        check(lib().synax_surrogate_save(self._h, str(path).encode()), "synax_surrogate_save")

    def load(self, path: str) -> None:
        check(lib().synax_surrogate_load(self._h, str(path).encode()), "synax_surrogate_load")

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().synax_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def surrogate_coeffs(sur: Surrogate, theta):
    """Differentiable coefficients: a torch.autograd.Function whose backward
    is the surrogate's own vector-Jacobian product (dL/dc -> dL/dtheta)."""
    import torch

    class _SurrogateCoeffs(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            ctx.save_for_backward(th)
            return sur(th.detach())

        @staticmethod
        def backward(ctx, gc):
            (th,) = ctx.saved_tensors
            _, gt = sur(th.detach(), gc)
            return gt.to(th.dtype)

    return _SurrogateCoeffs.apply(theta)
