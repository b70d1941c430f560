"""ctypes binding of libsynax (include/synax.h): argument marshalling only.

Every step of the march runs in the CUDA library; this module copies a
``Problem`` into the C struct, passes raw device pointers and the current
torch stream, and turns negative status codes into exceptions.  There is no
CPU fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libsynax.so")

SYNAX_OK = 0
SYNAX_EINVAL = -1
SYNAX_ENONFINITE = -2
SYNAX_ECUDA = -3
SYNAX_ENOMEM = -4
SYNAX_ETIMEOUT = -5
SYNAX_ENOTSUP = -6
SYNAX_ESPACE = -7
SYNAX_EBOUNDS = -8

SITE_MAP_STORE, SITE_SEED_LOAD, SITE_PARTIAL, SITE_GRID_LOAD, SITE_GRID_SCATTER, SITE_BATCH_SET, \
    SITE_GEMM_WAIT = range(1, 8)

PIPES = {"ffma": 0, "ffma2": 1, "ex2": 2, "lg2": 3, "sin": 4, "cos": 5, "rcp": 6, "rsqrt": 7, "frnd": 8, "f2i": 9}

SYNAX_F64 = 1 << 0
SYNAX_BOX_CLIP = 1 << 1
SYNAX_CHECKED = 1 << 2

MAX_FREQ = 16
MAX_THETA = 32


class SynaxError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


class SynaxProblem(ctypes.Structure):
    _fields_ = [
        ("nside", ctypes.c_int32),
        ("n_steps", ctypes.c_int32),
        ("r_max_kpc", ctypes.c_double),
        ("box_kpc", ctypes.c_double * 3),
        ("obs_kpc", ctypes.c_double * 3),
        ("n_freq", ctypes.c_int32),
        ("freq_hz", ctypes.c_double * MAX_FREQ),
        ("model_id", ctypes.c_int32),
        ("n_theta", ctypes.c_int32),
        ("theta", ctypes.c_double * MAX_THETA),
        ("flags", ctypes.c_uint32),
        ("rm_rule", ctypes.c_int32),
        ("pix_begin", ctypes.c_int64),
        ("pix_count", ctypes.c_int64),
        ("grid_dev", ctypes.c_void_p),
        ("grid_n", ctypes.c_int32 * 3),
        ("reserved", ctypes.c_int32),
    ]


#: Exported symbols of include/synax.h with (restype, argtypes).
class SynaxSurrogateCfg(ctypes.Structure):
    """Mirror of synax_surrogate_cfg (include/synax.h)."""
    _fields_ = [
        ("n_theta", ctypes.c_int32), ("width", ctypes.c_int32), ("depth", ctypes.c_int32),
        ("nside", ctypes.c_int32), ("n_basis", ctypes.c_int32), ("batch", ctypes.c_int32),
        ("max_eval", ctypes.c_int32), ("map_chunk", ctypes.c_int32), ("total_steps", ctypes.c_int32),
        ("basis_kind", ctypes.c_int32),
        ("lr", ctypes.c_double), ("lr_min", ctypes.c_double), ("beta1", ctypes.c_double),
        ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
        ("theta_lo", ctypes.c_double * 64), ("theta_hi", ctypes.c_double * 64),
        ("basis_sign", ctypes.POINTER(ctypes.c_int8)), ("basis_rows", ctypes.POINTER(ctypes.c_int32)),
    ]


class SynaxHmcCfg(ctypes.Structure):
    """Mirror of synax_hmc_cfg (include/synax.h)."""
    _fields_ = [
        ("n_leapfrog", ctypes.c_int32), ("step_size", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("inv_mass", ctypes.POINTER(ctypes.c_double)), ("lo", ctypes.POINTER(ctypes.c_double)),
        ("hi", ctypes.POINTER(ctypes.c_double)),
    ]


SUR_PARAMS, SUR_GRADS, SUR_ADAM_M, SUR_ADAM_V, SUR_NORM, SUR_LOSS = range(6)
SUR_BASIS_SRHT, SUR_BASIS_SH = 0, 1
_VP = ctypes.c_void_p

SIGNATURES = {
    "synax_forward": (ctypes.c_int, [ctypes.POINTER(SynaxProblem), ctypes.c_void_p, ctypes.c_void_p]),
    "synax_adjoint_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(SynaxProblem),
                                                     ctypes.POINTER(ctypes.c_size_t)]),
    "synax_adjoint": (ctypes.c_int, [ctypes.POINTER(SynaxProblem), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                     ctypes.c_void_p]),
    "synax_batch_plan_n_sets": (ctypes.c_int, [ctypes.c_void_p]),
    "synax_batch_plan_n_theta": (ctypes.c_int, [ctypes.c_void_p]),
    "synax_batch_plan_n_pairs": (ctypes.c_int, [ctypes.c_void_p]),
    "synax_set_batch_pairing": (ctypes.c_int, [ctypes.c_int]),
    "synax_batch_bind": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "synax_batch_run_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "synax_hmc_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "synax_hmc_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "synax_hmc_set": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]),
    "synax_hmc_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "synax_hmc_destroy": (None, [ctypes.c_void_p]),
    "synax_sh_basis": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "synax_grid_sample": (ctypes.c_int, [ctypes.POINTER(SynaxProblem), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "synax_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int64, ctypes.c_void_p]),
    "synax_adjoint_grid_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(SynaxProblem),
                                                          ctypes.POINTER(ctypes.c_size_t)]),
    "synax_adjoint_grid": (ctypes.c_int, [ctypes.POINTER(SynaxProblem), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_size_t, ctypes.c_void_p]),
    "synax_adjoint_noalloc": (ctypes.c_int, [ctypes.POINTER(SynaxProblem), ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "synax_eval_fields": (ctypes.c_int, [ctypes.POINTER(SynaxProblem), ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "synax_set_lanes_per_ray": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "synax_batch_plan_create": (ctypes.c_int, [ctypes.POINTER(SynaxProblem), ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_void_p)]),
    "synax_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "synax_batch_latencies": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "synax_batch_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "synax_batch_plan_destroy": (None, [ctypes.c_void_p]),
    "synax_gemm_bf16": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "synax_surrogate_create": (ctypes.c_int, [ctypes.POINTER(SynaxSurrogateCfg), ctypes.POINTER(_VP)]),
    "synax_surrogate_destroy": (None, [_VP]),
    "synax_surrogate_param_count": (ctypes.c_size_t, [_VP]),
    "synax_surrogate_set_params": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "synax_surrogate_get": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_size_t]),
    "synax_surrogate_set_normalization": (ctypes.c_int, [_VP, _VP, ctypes.c_float]),
    "synax_surrogate_project": (ctypes.c_int, [_VP, _VP, ctypes.c_longlong, _VP, _VP]),
    "synax_surrogate_dataset": (ctypes.c_int, [_VP, ctypes.POINTER(SynaxProblem), _VP, ctypes.c_longlong, _VP]),
    "synax_surrogate_step": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "synax_surrogate_train": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_uint64, _VP]),
    "synax_surrogate": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "synax_surrogate_judge": (ctypes.c_int, [_VP, ctypes.POINTER(SynaxProblem), _VP, ctypes.c_int, _VP,
                                             ctypes.c_double, _VP, _VP, _VP]),
    "synax_surrogate_gate": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "synax_surrogate_status": (ctypes.c_int, [_VP, _VP]),
    "synax_wait_selftest": (ctypes.c_int, [_VP, _VP, _VP]),
    "synax_surrogate_save": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "synax_surrogate_load": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "synax_pipe_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP,
                                       ctypes.POINTER(ctypes.c_longlong), _VP]),
    "synax_last_status": (ctypes.c_int, [_VP]),
    "synax_last_status_detail": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]),
    "synax_checked_selftest": (ctypes.c_int, []),
    "synax_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p]),
    "synax_last_cuda_error": (ctypes.c_int, []),
    "synax_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "synax_version": (ctypes.c_int, []),
}

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libsynax (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libsynax is not built ({LIB_PATH} missing); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` or "
                    "`python paper_2410_01136_gb300/cuda_build.py`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, what: str) -> None:
    if status == SYNAX_OK:
        return
    L = lib()
    msg = L.synax_strerror(status).decode()
    if status == SYNAX_ECUDA:
        msg += f" (cudaError {L.synax_last_cuda_error()})"
    raise SynaxError(status, f"{what}: {msg} [{status}]")


def problem_struct(prob) -> SynaxProblem:
    """Copy a Problem (paper_2410_01136_gb300.inputs.Problem or any object with
    the same fields) into the C struct."""
    s = SynaxProblem()
    s.nside = int(prob.nside)
    s.n_steps = int(prob.n_steps)
    s.r_max_kpc = float(prob.r_max_kpc)
    for k in range(3):
        s.box_kpc[k] = float(prob.box_kpc[k])
        s.obs_kpc[k] = float(prob.obs_kpc[k])
    freqs = list(prob.freq_hz)
    if len(freqs) > MAX_FREQ:
        raise ValueError(f"at most {MAX_FREQ} frequencies")
    s.n_freq = len(freqs)
    for k, f in enumerate(freqs):
        s.freq_hz[k] = float(f)
    s.model_id = int(prob.model_id)
    th = [float(x) for x in prob.theta]
    if len(th) > MAX_THETA:
        raise ValueError(f"at most {MAX_THETA} parameters")
    s.n_theta = len(th)
    for k, x in enumerate(th):
        s.theta[k] = x
    s.flags = (SYNAX_F64 if getattr(prob, "f64", False) else 0) | (
        SYNAX_BOX_CLIP if getattr(prob, "box_clip", False) else 0) | (
        SYNAX_CHECKED if getattr(prob, "checked", False) else 0)
    s.rm_rule = int(getattr(prob, "rm_rule", 0))
    s.pix_begin = int(getattr(prob, "pix_begin", 0))
    s.pix_count = int(getattr(prob, "pix_count", 0))
    grid = getattr(prob, "grid", None)
    if grid is not None:
        t = grid_device(prob)
        s.grid_dev = t.data_ptr()
        s.grid_n[0], s.grid_n[1], s.grid_n[2] = int(t.shape[2]), int(t.shape[1]), int(t.shape[0])
    return s


def grid_device(prob):
    """The grid model's node array on the current CUDA device in the march
    precision.  A device tensor is used as it is (it must be contiguous, of
    that dtype, [nz][ny][nx][3]); a host array is copied once and the copy is
    kept on the problem object (host grids of a Problem are read-only)."""
    import torch
    g = prob.grid
    dt = torch.float64 if getattr(prob, "f64", False) else torch.float32
    if isinstance(g, torch.Tensor):
        if not g.is_cuda or g.dtype != dt or not g.is_contiguous() or g.ndim != 4 or g.shape[3] != 3:
            raise ValueError(f"a device grid must be a contiguous CUDA {dt} tensor of shape [nz, ny, nx, 3]")
        return g
    key = (id(g), dt, torch.cuda.current_device())
    cached = getattr(prob, "_grid_device_copy", None)
    if cached is None or cached[0] != key:
        import numpy as np
        t = torch.as_tensor(np.array(g, copy=True)).to(device="cuda", dtype=dt).contiguous()   # host grids are read-only
        cached = (key, t)
        object.__setattr__(prob, "_grid_device_copy", cached)
    return cached[1]
