"""GB300-native synchrotron ray march (synax, arXiv 2410.01136).

Python surface of libsynax (include/synax.h).  PyTorch provides device memory
and streams; every step of the march runs in the library's CUDA kernels.

    from paper_2410_01136_gb300 import forward, adjoint, SynaxMaps, inputs
    prob = inputs.config2()
    maps = forward(prob)                 # [F, 3, n_pix] on the current CUDA device

There is no CPU path: without the built library (``build()``) or without a
CUDA device every call raises.
"""
from __future__ import annotations

import ctypes

from . import inputs
from . import _native
from ._native import (SYNAX_F64, SynaxError, check, lib, problem_struct)

__all__ = ["forward", "adjoint", "adjoint_grid", "adjoint_grid_workspace_bytes", "grid_sample", "adam_step", "GridFit", "HMC", "eval_fields", "BatchPlan", "adjoint_workspace_bytes", "SynaxMaps", "inputs", "build",
           "SynaxError", "last_status", "pipe_peaks", "set_lanes_per_ray", "set_batch_pairing"]


def build(force: bool = False, verbose: bool = False) -> str:
    from .cuda_build import build as _build
    return _build(force=force, verbose=verbose)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libsynax needs a CUDA device; none is available")
    return torch


def _stream_handle(torch, stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(int(s.cuda_stream))


def _map_dtype(torch, prob):
    return torch.float64 if getattr(prob, "f64", False) else torch.float32


def _check_map_tensor(torch, t, prob, name):
    shape = (prob.n_freq, 3, prob.n_pix_out)
    if not t.is_cuda or t.dtype != _map_dtype(torch, prob) or tuple(t.shape) != shape \
            or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {_map_dtype(torch, prob)} tensor of "
                         f"shape {shape}")


def forward(prob, out=None, stream=None):
    """March all pixels of `prob` (Sec. 2.3) and return the [F, 3, n_pix]
    brightness-temperature maps (I, Q, U) as a CUDA tensor."""
    torch = _torch()
    if out is None:
        out = torch.empty((prob.n_freq, 3, prob.n_pix_out), dtype=_map_dtype(torch, prob),
                          device="cuda")
    else:
        _check_map_tensor(torch, out, prob, "out")
    s = problem_struct(prob)
    check(lib().synax_forward(ctypes.byref(s), ctypes.c_void_p(out.data_ptr()),
                              _stream_handle(torch, stream)), "synax_forward")
    return out


def eval_fields(prob, pos, t, stream=None):
    """B (uG), N0, n_e (cm^-3) of prob's model at positions pos [n, 3] (kpc) with
    observer distances t [n], evaluated by the march's device code; returns a
    [n, 5] float64 CUDA tensor."""
    torch = _torch()
    pos = torch.as_tensor(pos, dtype=torch.float64, device="cuda").reshape(-1, 3).contiguous()
    t = torch.as_tensor(t, dtype=torch.float64, device="cuda").reshape(-1).contiguous()
    out = torch.empty((pos.shape[0], 5), dtype=torch.float64, device="cuda")
    s = problem_struct(prob)
    check(lib().synax_eval_fields(ctypes.byref(s), ctypes.c_void_p(pos.data_ptr()),
                                  ctypes.c_void_p(t.data_ptr()), pos.shape[0],
                                  ctypes.c_void_p(out.data_ptr()), _stream_handle(torch, stream)),
          "synax_eval_fields")
    return out


def adjoint_workspace_bytes(prob) -> int:
    s = problem_struct(prob)
    n = ctypes.c_size_t(0)
    check(lib().synax_adjoint_workspace_bytes(ctypes.byref(s), ctypes.byref(n)),
          "synax_adjoint_workspace_bytes")
    return int(n.value)


def adjoint(prob, gmaps=None, target=None, sigma: float = 1.0, maps_out=None, workspace=None,
            stream=None):
    """Gradient with respect to theta (a float64 CUDA tensor of n_theta values).

    VJP mode (gmaps given): sum(gmaps * dM/dtheta).  chi^2 mode (target given):
    d chi^2 / d theta with chi^2 = sum((M - target)^2) / sigma^2; returns
    (grad, chi2) in that mode.  maps_out optionally receives M.
    """
    torch = _torch()
    if (gmaps is None) == (target is None):
        raise ValueError("give exactly one of gmaps (VJP mode) or target (chi^2 mode)")
    seed = gmaps if gmaps is not None else target
    _check_map_tensor(torch, seed, prob, "gmaps" if gmaps is not None else "target")
    if maps_out is not None:
        _check_map_tensor(torch, maps_out, prob, "maps_out")
    nbytes = adjoint_workspace_bytes(prob)
    if workspace is None:
        workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
    grad = torch.empty(len(prob.theta), dtype=torch.float64, device="cuda")
    chi2 = torch.empty(1, dtype=torch.float64, device="cuda") if target is not None else None
    s = problem_struct(prob)
    check(lib().synax_adjoint(
        ctypes.byref(s),
        ctypes.c_void_p(gmaps.data_ptr() if gmaps is not None else 0),
        ctypes.c_void_p(target.data_ptr() if target is not None else 0),
        ctypes.c_double(float(sigma)),
        ctypes.c_void_p(grad.data_ptr()),
        ctypes.c_void_p(chi2.data_ptr() if chi2 is not None else 0),
        ctypes.c_void_p(maps_out.data_ptr() if maps_out is not None else 0),
        ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()),
        _stream_handle(torch, stream)), "synax_adjoint")
    if target is not None:
        return grad, chi2
    return grad


def adjoint_grid_workspace_bytes(prob) -> int:
    s = problem_struct(prob)
    n = ctypes.c_size_t(0)
    check(lib().synax_adjoint_grid_workspace_bytes(ctypes.byref(s), ctypes.byref(n)),
          "synax_adjoint_grid_workspace_bytes")
    return int(n.value)


def adjoint_grid(prob, gmaps=None, target=None, sigma: float = 1.0, maps_out=None, grid_grad=None,
                 workspace=None, stream=None):
    """Grid model (Sec. 3.3): the gradient with respect to theta = [N0_obs, p,
    ne0] and to every grid value.  Modes as in ``adjoint``; returns
    (grad, grid_grad) in VJP mode and (grad, grid_grad, chi2) in chi^2 mode,
    grid_grad a CUDA tensor shaped like the grid ([nz, ny, nx, 3]).  The
    grid gradient is summed with atomic adds (not bitwise reproducible)."""
    torch = _torch()
    if (gmaps is None) == (target is None):
        raise ValueError("give exactly one of gmaps (VJP mode) or target (chi^2 mode)")
    if getattr(prob, "grid", None) is None:
        raise ValueError("adjoint_grid needs a grid-model problem")
    seed = gmaps if gmaps is not None else target
    _check_map_tensor(torch, seed, prob, "gmaps" if gmaps is not None else "target")
    if maps_out is not None:
        _check_map_tensor(torch, maps_out, prob, "maps_out")
    s = problem_struct(prob)
    shape = (s.grid_n[2], s.grid_n[1], s.grid_n[0], 3)
    if grid_grad is None:
        grid_grad = torch.empty(shape, dtype=_map_dtype(torch, prob), device="cuda")
    elif (not grid_grad.is_cuda or grid_grad.dtype != _map_dtype(torch, prob)
          or tuple(grid_grad.shape) != shape or not grid_grad.is_contiguous()):
        raise ValueError(f"grid_grad must be a contiguous CUDA {_map_dtype(torch, prob)} tensor of shape {shape}")
    nbytes = ctypes.c_size_t(0)
    check(lib().synax_adjoint_grid_workspace_bytes(ctypes.byref(s), ctypes.byref(nbytes)),
          "synax_adjoint_grid_workspace_bytes")
    if workspace is None:
        workspace = torch.empty(max(nbytes.value, 1), dtype=torch.uint8, device="cuda")
    grad = torch.empty(len(prob.theta), dtype=torch.float64, device="cuda")
    chi2 = torch.empty(1, dtype=torch.float64, device="cuda") if target is not None else None
    check(lib().synax_adjoint_grid(
        ctypes.byref(s),
        ctypes.c_void_p(gmaps.data_ptr() if gmaps is not None else 0),
        ctypes.c_void_p(target.data_ptr() if target is not None else 0),
        ctypes.c_double(float(sigma)),
        ctypes.c_void_p(grad.data_ptr()),
        ctypes.c_void_p(chi2.data_ptr() if chi2 is not None else 0),
        ctypes.c_void_p(maps_out.data_ptr() if maps_out is not None else 0),
        ctypes.c_void_p(grid_grad.data_ptr()),
        ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()),
        _stream_handle(torch, stream)), "synax_adjoint_grid")
    if target is not None:
        return grad, grid_grad, chi2
    return grad, grid_grad


def grid_sample(prob, n, stream=None):
    """B of prob's analytic model at the nodes of an n = (n_x, n_y, n_z) grid
    spanning prob's box (synax_grid_sample); returns a [n_z, n_y, n_x, 3] CUDA
    tensor in the march precision, ready to be a grid model's ``grid``."""
    torch = _torch()
    nx, ny, nz = (int(v) for v in n)
    out = torch.empty((nz, ny, nx, 3), dtype=_map_dtype(torch, prob), device="cuda")
    gn = (ctypes.c_int32 * 3)(nx, ny, nz)
    s = problem_struct(prob)
    check(lib().synax_grid_sample(ctypes.byref(s), gn, ctypes.c_void_p(out.data_ptr()),
                                  _stream_handle(torch, stream)), "synax_grid_sample")
    return out


def adam_step(params, grads, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8, stream=None):
    """One in-place Adam step on contiguous float32 CUDA tensors (synax_adam)."""
    torch = _torch()
    for name, x in (("params", params), ("grads", grads), ("m", m), ("v", v)):
        if not x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous() or x.numel() != params.numel():
            raise ValueError(f"{name} must be a contiguous CUDA float32 tensor of {params.numel()} values")
    check(lib().synax_adam(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(grads.data_ptr()),
                           ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()), params.numel(),
                           float(lr), float(beta1), float(beta2), float(eps), int(t),
                           _stream_handle(torch, stream)), "synax_adam")


class GridFit:
    """Field-level fit of a grid model to a target map (Sec. 3.3): every step
    is synax_adjoint_grid in chi^2 mode (maps, chi^2, grid gradient) followed
    by synax_adam on the grid, all enqueued on one stream; buffers are
    allocated once.

        fit = GridFit(prob, target, sigma, lr=0.05)   # prob.grid: the start
        chi2 = fit.run(200)                           # chi^2 before each step
        fit.grid                                      # the fitted grid (CUDA tensor)
    """

    def __init__(self, prob, target, sigma: float, lr: float = 0.05, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8):
        torch = _torch()
        if getattr(prob, "f64", False):
            raise ValueError("GridFit runs the FP32 march (synax_adam is float32)")
        from ._native import grid_device
        self.grid = grid_device(prob).clone()
        self.prob = prob.replace(grid=self.grid)
        _check_map_tensor(torch, target, self.prob, "target")
        self.target, self.sigma = target, float(sigma)
        self.lr, self.beta1, self.beta2, self.eps = lr, beta1, beta2, eps
        self.m = torch.zeros_like(self.grid)
        self.v = torch.zeros_like(self.grid)
        self.g = torch.empty_like(self.grid)
        self.maps = torch.empty_like(target)
        self.workspace = torch.empty(max(adjoint_grid_workspace_bytes(self.prob), 1), dtype=torch.uint8,
                                     device="cuda")
        self.t = 0

    def step(self):
        """One chi^2 + gradient evaluation and Adam update; returns chi^2 (a
        device scalar) of the grid before the update."""
        _, _, chi2 = adjoint_grid(self.prob, target=self.target, sigma=self.sigma, maps_out=self.maps,
                                  grid_grad=self.g, workspace=self.workspace)
        self.t += 1
        adam_step(self.grid, self.g, self.m, self.v, self.t, self.lr, self.beta1, self.beta2, self.eps)
        return chi2

    def run(self, n_steps: int):
        torch = _torch()
        out = torch.empty(n_steps, dtype=torch.float64, device="cuda")
        for k in range(n_steps):
            out[k:k + 1].copy_(self.step())
        return out


class BatchPlan:
    """A persistent, graph-captured batch of map+gradient evaluations
    (synax_batch_* of include/synax.h): one launch for many parameter sets of
    uneven Nside and step count.

        plan = BatchPlan(problems)                    # allocates once
        grads, chi2 = plan.run(targets=[...], sigma=0.5, thetas=new_thetas)
        plan.latencies()                              # per-set completion, ms
    """

    def __init__(self, problems):
        self.problems = list(problems)
        n = len(self.problems)
        arr = (_native.SynaxProblem * max(n, 1))()
        for i, p in enumerate(self.problems):
            arr[i] = problem_struct(p)
        self._n = n
        self._n_theta = len(self.problems[0].theta) if n else 0
        h = ctypes.c_void_p()
        check(lib().synax_batch_plan_create(arr, n, ctypes.byref(h)), "synax_batch_plan_create")
        self._h = h

    def info(self) -> dict:
        nt = ctypes.c_longlong()
        lpr = ctypes.c_int()
        grid = ctypes.c_int()
        check(lib().synax_batch_plan_info(self._h, ctypes.byref(nt), ctypes.byref(lpr), ctypes.byref(grid)),
              "synax_batch_plan_info")
        return {"n_tiles": nt.value, "lanes_per_ray": lpr.value, "grid": grid.value,
                "n_pairs": lib().synax_batch_plan_n_pairs(self._h)}

    def run(self, targets=None, seeds=None, sigma: float = 1.0, thetas=None, maps=None, grads=None,
            chi2=None, stream=None):
        """chi^2 mode (targets) or VJP mode (seeds): lists of per-set CUDA tensors
        [F, 3, n_pix_s].  thetas: [n_sets, n_theta] array or None to keep the
        previous parameters.  Returns (grads [n_sets, n_theta], chi2 [n_sets])
        as CUDA float64 tensors (chi2 is None in VJP mode)."""
        import numpy as np
        torch = _torch()
        if (targets is None) == (seeds is None):
            raise ValueError("give exactly one of targets (chi^2) or seeds (VJP)")
        src = targets if targets is not None else seeds
        if len(src) != self._n:
            raise ValueError("one target/seed map per set")
        for t, p in zip(src, self.problems):
            _check_map_tensor(torch, t, p, "target/seed")
        if maps is not None:
            for t, p in zip(maps, self.problems):
                if t is not None:
                    _check_map_tensor(torch, t, p, "maps")
        if grads is None:
            grads = torch.empty((self._n, self._n_theta), dtype=torch.float64, device="cuda")
        if chi2 is None and targets is not None:
            chi2 = torch.empty(self._n, dtype=torch.float64, device="cuda")
        th_ptr = None
        if thetas is not None:
            th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(self._n, self._n_theta))
            self._thetas = th
            for i in range(self._n):
                self.problems[i] = self.problems[i].with_theta(th[i])
            th_ptr = th.ctypes.data_as(ctypes.c_void_p)
        seed_arr = (ctypes.c_void_p * self._n)(*[t.data_ptr() for t in src])
        map_arr = None
        if maps is not None:
            map_arr = (ctypes.c_void_p * self._n)(*[(t.data_ptr() if t is not None else None) for t in maps])
        check(lib().synax_batch(self._h, th_ptr, seed_arr, 0 if targets is not None else 1,
                                ctypes.c_double(float(sigma)), map_arr,
                                ctypes.c_void_p(grads.data_ptr()),
                                ctypes.c_void_p(chi2.data_ptr() if chi2 is not None else 0),
                                _stream_handle(torch, stream)), "synax_batch")
        return grads, chi2

    def bind(self, targets=None, seeds=None, sigma: float = 1.0, maps=None, grads=None, chi2=None):
        """Fixes seeds/targets, sigma and outputs for run_device (synax_batch_bind);
        returns (grads [n_sets, n_theta], chi2 [n_sets] or None), the tensors
        every later run_device writes."""
        torch = _torch()
        if (targets is None) == (seeds is None):
            raise ValueError("give exactly one of targets (chi^2) or seeds (VJP)")
        src = targets if targets is not None else seeds
        if len(src) != self._n:
            raise ValueError("one target/seed map per set")
        for t, p in zip(src, self.problems):
            _check_map_tensor(torch, t, p, "target/seed")
        if grads is None:
            grads = torch.empty((self._n, self._n_theta), dtype=torch.float64, device="cuda")
        if chi2 is None and targets is not None:
            chi2 = torch.empty(self._n, dtype=torch.float64, device="cuda")
        seed_arr = (ctypes.c_void_p * self._n)(*[t.data_ptr() for t in src])
        map_arr = None
        if maps is not None:
            map_arr = (ctypes.c_void_p * self._n)(*[(t.data_ptr() if t is not None else None) for t in maps])
        check(lib().synax_batch_bind(self._h, seed_arr, 0 if targets is not None else 1, ctypes.c_double(float(sigma)),
                                     map_arr, ctypes.c_void_p(grads.data_ptr()),
                                     ctypes.c_void_p(chi2.data_ptr() if chi2 is not None else 0)),
              "synax_batch_bind")
        self._bound = (list(src), maps, grads, chi2)          # the plan reads these on every run
        return grads, chi2

    def run_device(self, theta, stream=None):
        """Runs the bound batch with theta [n_sets, n_theta] (CUDA float64)
        read on the device (synax_batch_run_device)."""
        torch = _torch()
        if not theta.is_cuda or theta.dtype != torch.float64 or not theta.is_contiguous() \
                or tuple(theta.shape) != (self._n, self._n_theta):
            raise ValueError(f"theta must be a contiguous CUDA float64 tensor [{self._n}, {self._n_theta}]")
        self._theta_dev = theta
        check(lib().synax_batch_run_device(self._h, ctypes.c_void_p(theta.data_ptr()), _stream_handle(torch, stream)),
              "synax_batch_run_device")

    def latencies(self):
        import numpy as np
        out = np.zeros(self._n, dtype=np.float64)
        check(lib().synax_batch_latencies(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
              "synax_batch_latencies")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().synax_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_batch_pairing(on: bool) -> None:
    """Whether batch plans created afterwards march sets of one ray geometry
    two at a time (the default) or every set alone."""
    check(lib().synax_set_batch_pairing(1 if on else 0), "synax_set_batch_pairing")


def set_lanes_per_ray(lanes: int, n_steps_min: int = -1) -> None:
    """Launch tuning: 8, 16 or 32 lanes per ray (0 = built-in rule), for every
    map (n_steps_min < 0) or for the step-count bin containing n_steps_min."""
    check(lib().synax_set_lanes_per_ray(int(n_steps_min), int(lanes)), "synax_set_lanes_per_ray")


def last_status(stream=None) -> tuple[int, int, int]:
    """(code, site, index) of the first device-side error recorded since the
    last read (synax_last_status, which synchronises the stream and clears
    the word): code 0 when none, SYNAX_EBOUNDS from a SYNAX_CHECKED launch,
    SYNAX_ETIMEOUT from a bounded wait that gave up."""
    torch = _torch()
    code = lib().synax_last_status(_stream_handle(torch, stream))
    if code == _native.SYNAX_ECUDA:
        check(code, "synax_last_status")
    site, index = ctypes.c_int(0), ctypes.c_longlong(0)
    lib().synax_last_status_detail(ctypes.byref(site), ctypes.byref(index))
    return code, site.value, index.value


def pipe_peaks(pipes=("ffma", "ffma2", "ex2", "lg2", "sin", "cos", "rcp", "rsqrt", "frnd", "f2i"), blocks_per_sm: int = 8,
               iters: int = 4096, repeats: int = 5) -> dict:
    """Measured throughput of the FP32 pipe and the SFU on the current device
    (synax_pipe_peak): per pipe the best of `repeats` launches, in element
    operations per second, from CUDA events on the launching stream.  A grid
    of blocks_per_sm 256-thread CTAs per SM keeps every SM's pipes full."""
    torch = _torch()
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = blocks_per_sm * sms
    sink = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    h = _stream_handle(torch, stream)
    ops = ctypes.c_longlong(0)
    out = {}
    for name in pipes:
        code = _native.PIPES[name]
        check(lib().synax_pipe_peak(code, blocks, 64, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops), h),
              "synax_pipe_peak")                                   # warm-up
        best = 0.0
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            check(lib().synax_pipe_peak(code, blocks, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops),
                                        h), "synax_pipe_peak")
            b.record(stream)
            b.synchronize()
            best = max(best, ops.value / (a.elapsed_time(b) * 1e-3))
        out[name] = best
    out["sms"] = sms
    return out


class SynaxMaps:
    """torch.autograd.Function over the march: maps = SynaxMaps.apply(theta, prob).

    theta: float64 tensor (CPU or CUDA) of the model parameters; the maps come
    back on the current CUDA device.  backward() calls the library's adjoint
    in VJP mode with the incoming map gradient.
    """

    _fn = None

    @classmethod
    def apply(cls, theta, prob):
        if cls._fn is None:
            cls._fn = _make_function()
        return cls._fn.apply(theta, prob)


def _make_function():
    import torch

    class _SynaxMapsFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, prob):
            th = theta.detach().to("cpu", torch.float64).numpy()
            p = prob.with_theta(th)
            ctx.prob = p
            ctx.theta_device = theta.device
            return forward(p)

        @staticmethod
        def backward(ctx, gmaps):
            g = adjoint(ctx.prob, gmaps=gmaps.contiguous())
            return g.to(ctx.theta_device), None

    return _SynaxMapsFn


from .hmc import HMC, effective_sample_size, laplace_inv_mass  # noqa: E402  (uses BatchPlan above)
