"""FP64 CPU oracle of the synax ray march -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls it, and this package never
imports the product.  Both sides receive the same seeded inputs from
``paper_2410_01136_gb300.inputs``, which holds no arithmetic of the method.

The arithmetic lives in ``synax_oracle.c`` (plain C, double precision,
pixel -> step -> frequency loops; see the header of that file for the
definition it follows: Sec. 2.1-2.3 of the paper, Eq. 2, 5-9).  This module
compiles it with gcc, loads it with ctypes and adds two plain-numpy helpers:
the Gaussian chi^2 of Sec. 3.1 (Eq. 15, up to the factor -1/2) and central
finite differences, the gradient reference for the adjoint.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, textbook forms, invariants, brute force).  The JF12-type field
model is defined by this project (after Jansson & Farrar 2012), so no
published values pin it; its evaluation is pinned by properties the
definition implies (``tests/test_oracle_jf12.py``: a divergence-free disc
and halo, the disc's pitch, the arm weights' partition of unity, the arm
layout and winding, the X field's lines and flux, the densities); the
WMAP-type field by Eq. 13's direction, its symmetry, the uniform x field and
its densities (``tests/test_oracle_wmap.py``).  The grid model's interpolation is pinned by exactness on multilinear
fields, by scipy's linear grid interpolator and by node values
(``tests/test_oracle_grid.py``); the stacked WMAP model of Sec. 4.3 by the
magnitude, pitch and elevation of each of its Eq. 13 components and its
stacking (``tests/test_oracle_wmap_stack.py``).  ``oracle/hmc.py`` holds a
plain HMC (Neal 2011) with the library's documented random numbers, pinned by
the exactness of its leapfrog on a Gaussian and by sampling moments
(``tests/test_oracle_hmc.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synax_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

MODEL_TOY, MODEL_WMAP, MODEL_JF12, MODEL_GRID, MODEL_WMAP_STACK = 0, 1, 2, 3, 4
N_THETA = {MODEL_TOY: 7, MODEL_WMAP: 8, MODEL_JF12: 16, MODEL_GRID: 3, MODEL_WMAP_STACK: 19}


class _OracleProblem(ctypes.Structure):
    _fields_ = [
        ("nside", ctypes.c_int32),
        ("n_steps", ctypes.c_int32),
        ("r_max_kpc", ctypes.c_double),
        ("box_clip", ctypes.c_int32),
        ("box_kpc", ctypes.c_double * 3),
        ("obs_kpc", ctypes.c_double * 3),
        ("n_freq", ctypes.c_int32),
        ("freq_hz", ctypes.c_double * 16),
        ("model_id", ctypes.c_int32),
        ("n_theta", ctypes.c_int32),
        ("theta", ctypes.c_double * 32),
        ("rm_rule", ctypes.c_int32),
        ("grid", ctypes.POINTER(ctypes.c_double)),
        ("grid_n", ctypes.c_int32 * 3),
    ]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synax_oracle.c into _build/liboracle.so (IEEE double, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-fPIC", "-shared",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_healpix_centre.argtypes = [ctypes.c_int64, ctypes.c_int64,
                                                  ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_double)]
            lib.oracle_healpix_centre.restype = ctypes.c_int
            lib.oracle_los.argtypes = [ctypes.c_int64, ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_double)]
            lib.oracle_los.restype = ctypes.c_int
            lib.oracle_fields.argtypes = [ctypes.POINTER(_OracleProblem),
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
            lib.oracle_fields.restype = ctypes.c_int
            lib.oracle_emissivity.argtypes = [ctypes.c_double] * 4 + [
                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            lib.oracle_emissivity.restype = None
            lib.oracle_rm_constant.argtypes = []
            lib.oracle_rm_constant.restype = ctypes.c_double
            lib.oracle_brightness_temperature.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.oracle_brightness_temperature.restype = ctypes.c_double
            lib.oracle_forward.argtypes = [ctypes.POINTER(_OracleProblem),
                                           ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_int]
            lib.oracle_forward.restype = ctypes.c_int
            lib.oracle_fields_batch.argtypes = [ctypes.POINTER(_OracleProblem), ctypes.c_int64,
                                                ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_double)]
            lib.oracle_fields_batch.restype = ctypes.c_int
            lib.oracle_ray_length.argtypes = [ctypes.POINTER(_OracleProblem), ctypes.c_int64]
            lib.oracle_ray_length.restype = ctypes.c_double
            lib.oracle_grid_interp.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double)]
            lib.oracle_grid_interp.restype = None
            _lib = lib
    return _lib


def _to_struct(prob) -> _OracleProblem:
    """Copy a problem description (any object with the fields below) into the
    oracle's own C struct."""
    s = _OracleProblem()
    s.nside = int(prob.nside)
    s.n_steps = int(prob.n_steps)
    s.r_max_kpc = float(prob.r_max_kpc)
    s.box_clip = 1 if prob.box_clip else 0
    for k in range(3):
        s.box_kpc[k] = float(prob.box_kpc[k])
        s.obs_kpc[k] = float(prob.obs_kpc[k])
    freqs = list(prob.freq_hz)
    if not 1 <= len(freqs) <= 16:
        raise ValueError("1..16 frequencies")
    s.n_freq = len(freqs)
    for k, f in enumerate(freqs):
        s.freq_hz[k] = float(f)
    s.model_id = int(prob.model_id)
    th = [float(x) for x in prob.theta]
    if len(th) > 32:
        raise ValueError("at most 32 parameters")
    s.n_theta = len(th)
    for k, x in enumerate(th):
        s.theta[k] = x
    s.rm_rule = int(getattr(prob, "rm_rule", 0))
    grid = getattr(prob, "grid", None)
    if grid is not None:
        g = np.ascontiguousarray(np.asarray(grid, dtype=np.float64))
        if g.ndim != 4 or g.shape[3] != 3 or min(g.shape[:3]) < 2:
            raise ValueError("grid must be [nz][ny][nx][3] with every n >= 2")
        s._grid_keepalive = g              # the struct points into this array
        s.grid = g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        s.grid_n[0], s.grid_n[1], s.grid_n[2] = g.shape[2], g.shape[1], g.shape[0]
    return s


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def forward(prob, pix=None, threads: int | None = None) -> np.ndarray:
    """Brightness-temperature maps, shape [F, 3, n] (I, Q, U), float64.

    pix: None for the full RING-ordered map, else an array of pixel indices.
    """
    lib = _load()
    s = _to_struct(prob)
    npix_all = 12 * s.nside * s.nside
    if pix is None:
        n = npix_all
        pix_ptr = None
    else:
        pix_arr = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
        n = int(pix_arr.size)
        pix_ptr = pix_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    out = np.zeros((s.n_freq, 3, n), dtype=np.float64)
    if n == 0:
        return out
    rc = lib.oracle_forward(ctypes.byref(s), pix_ptr, n,
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            int(threads or default_threads()))
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return out


def healpix_centre(nside: int, pix: int) -> tuple[float, float]:
    """(z = cos colatitude, phi) of a RING pixel centre."""
    z = ctypes.c_double()
    phi = ctypes.c_double()
    if _load().oracle_healpix_centre(nside, pix, ctypes.byref(z), ctypes.byref(phi)) != 0:
        raise ValueError("bad pixel")
    return z.value, phi.value


def los(nside: int, pix: int) -> dict:
    """LOS triad of one pixel: n, e_l, e_b (unit vectors) and (l, b) in rad."""
    out = (ctypes.c_double * 11)()
    if _load().oracle_los(nside, pix, out) != 0:
        raise ValueError("bad pixel")
    a = np.array(out[:], dtype=np.float64)
    return {"n": a[0:3], "el": a[3:6], "eb": a[6:9], "l": a[9], "b": a[10]}


def ray_length(prob, pix: int) -> float:
    s = _to_struct(prob)
    return float(_load().oracle_ray_length(ctypes.byref(s), pix))


def grid_interp(grid, box_kpc, r) -> np.ndarray:
    """Trilinear B (uG) of a cell-centred grid [nz][ny][nx][3] over the box at r (kpc)."""
    g = np.ascontiguousarray(np.asarray(grid, dtype=np.float64))
    n = (ctypes.c_int32 * 3)(g.shape[2], g.shape[1], g.shape[0])
    box = (ctypes.c_double * 3)(*[float(x) for x in box_kpc])
    rr = (ctypes.c_double * 3)(*[float(x) for x in r])
    B = (ctypes.c_double * 3)()
    _load().oracle_grid_interp(g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n, box, rr, B)
    return np.array(B[:])


def fields(prob, r, t: float = 0.0):
    """(B [uG, 3], N0 [cm^-3], n_e [cm^-3]) of the problem's model at r (kpc).
    t is the distance from the observer (toy model sphere only)."""
    s = _to_struct(prob)
    rr = (ctypes.c_double * 3)(*[float(x) for x in r])
    B = (ctypes.c_double * 3)()
    n0 = ctypes.c_double()
    ne = ctypes.c_double()
    if _load().oracle_fields(ctypes.byref(s), rr, float(t), B, ctypes.byref(n0), ctypes.byref(ne)) != 0:
        raise ValueError("bad model")
    return np.array(B[:]), n0.value, ne.value


def fields_batch(prob, r, t) -> np.ndarray:
    """Fields at many points: r [n, 3] kpc, t [n] observer distances ->
    [n, 5] = (Bx, By, Bz, N0, n_e)."""
    s = _to_struct(prob)
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(-1, 3))
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(-1))
    out = np.zeros((r.shape[0], 5), dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    if _load().oracle_fields_batch(ctypes.byref(s), r.shape[0], r.ctypes.data_as(dp),
                                   t.ctypes.data_as(dp), out.ctypes.data_as(dp)) != 0:
        raise ValueError("bad model")
    return out


def emissivity(nu: float, p: float, b_trans_gauss: float, n0: float) -> tuple[float, float]:
    """(j_I, j_P) of Eq. 2 and Eq. 5 in cgs (erg s^-1 cm^-3 Hz^-1 sr^-1)."""
    jI = ctypes.c_double()
    jP = ctypes.c_double()
    _load().oracle_emissivity(float(nu), float(p), float(b_trans_gauss), float(n0),
                              ctypes.byref(jI), ctypes.byref(jP))
    return jI.value, jP.value


def rm_constant() -> float:
    """q_e^3 / (2 pi m_e^2 c^4) of Eq. 7, cgs."""
    return float(_load().oracle_rm_constant())


def brightness_temperature(I: float, nu: float) -> float:
    return float(_load().oracle_brightness_temperature(float(I), float(nu)))


def chi2(maps: np.ndarray, target: np.ndarray, sigma: float) -> float:
    """chi^2 = sum over all map entries of (M - T)^2 / sigma^2, i.e. -2 log L
    of Sec. 3.1 (Eq. 15) up to its constant, summed over I, Q and U and all
    frequencies."""
    d = np.asarray(maps, dtype=np.float64) - np.asarray(target, dtype=np.float64)
    return float(np.sum(d * d) / (sigma * sigma))


def fd_gradient(loss, theta, steps) -> np.ndarray:
    """Central finite differences (loss(theta + h e_i) - loss(theta - h e_i)) / 2h
    for every component, h = steps[i]."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros_like(theta)
    for i in range(theta.size):
        h = float(steps[i])
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        g[i] = (loss(tp) - loss(tm)) / (2.0 * h)
    return g
