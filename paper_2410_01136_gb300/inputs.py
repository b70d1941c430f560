"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds no arithmetic of the method: only a counter-based random
generator, the problem description and the recipes of the synthetic
workloads (sizes, frequencies, parameter draws).  Both the CUDA binding and
the oracle read a ``Problem``; neither is imported here.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated as a counter-based
generator: value i of stream s is mix64(s + (i + 1) * 0x9E3779B97F4A7C15).
Uniforms take the top 53 bits; normals use the Box-Muller transform.  The
stream is the same on every machine and numpy version.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MODEL_TOY, MODEL_WMAP, MODEL_JF12, MODEL_GRID, MODEL_WMAP_STACK = 0, 1, 2, 3, 4
N_THETA = {MODEL_TOY: 7, MODEL_WMAP: 8, MODEL_JF12: 16, MODEL_GRID: 3, MODEL_WMAP_STACK: 19}

#: Parameter names of each model, in theta order.
THETA_NAMES = {
    MODEL_TOY: ["Bx", "By", "Bz", "ne", "N0", "p", "R0"],
    MODEL_WMAP: ["b0", "psi0", "psi1", "chi0B", "Bux", "N0_obs", "p", "ne0"],
    MODEL_JF12: [f"b{k + 1}" for k in range(8)]
    + ["B_h", "z_h", "B_X", "theta_X", "N0_obs", "p", "h1", "h2"],
    MODEL_GRID: ["N0_obs", "p", "ne0"],
    MODEL_WMAP_STACK: [f"{n}_{k}" for k in range(1, 5) for n in ("b0", "psi0", "psi1", "chi0B")]
    + ["N0_obs", "p", "ne0"],
}

#: Index of the CR spectral index p in each model's theta.
P_INDEX = {MODEL_TOY: 5, MODEL_WMAP: 6, MODEL_JF12: 13, MODEL_GRID: 1, MODEL_WMAP_STACK: 17}

OBS_PAPER_KPC = (-8.3, 0.0, 0.006)      # Sec. 2.1
OBS_CONFIG_KPC = (-8.5, 0.0, 0.015)     # synthetic workloads
BOX_PAPER_KPC = (40.0, 40.0, 10.0)      # Sec. 2.4
GRID_PAPER_N = (128, 128, 32)           # B grid nodes (nx, ny, nz), Sec. 3.3
N0_EARTH = 4.0e-5                       # cm^-3, Sec. 3.1

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n consecutive SplitMix64 outputs of stream `seed`, starting at index `offset`."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        return _mix64(state)


def substream(seed: int, tag: int) -> int:
    """A seed for an independent sub-stream (one mix of seed and tag)."""
    with np.errstate(over="ignore"):
        v = np.array([(seed * 0x100000001B3 + tag) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return int(_mix64(v)[0])


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    u = (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller over pairs of uniforms."""
    m = (n + 1) // 2
    raw = splitmix64(seed, 2 * m)
    u1 = ((raw[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
    u2 = (raw[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m, dtype=np.float64)
    out[0::2] = rad * np.cos(2.0 * math.pi * u2)
    out[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return out[:n]


@dataclasses.dataclass
class Problem:
    """One map to march (the paper's problem statement, Sec. 2.3).

    nside, n_steps: HEALPix resolution and N_int.  freq_hz: 1..16
    frequencies.  model_id / theta: field model and its parameters (see
    THETA_NAMES).  r_max_kpc: ray length, unless box_clip, in which case each
    ray ends at the boundary of the box box_kpc centred on the Galactic centre.
    obs_kpc: observer position.  f64: march in double precision and return
    double maps.  pix_begin / pix_count: a contiguous RING pixel range
    (pix_count 0 = to the end of the map).  rm_rule: how much of a cell's
    own n_e B_LOS dr enters the RM at its midpoint: 0 half (default), 1 none,
    2 all of it (a plain cumulative sum).  grid: the grid model's B nodes,
    [nz][ny][nx][3] in uG, spanning box_kpc wall to wall (grid model only):
    a host array (kept as a read-only float64 copy) or a device tensor of the
    march precision, used in place.  checked: launch the bounds-checked
    kernels (SYNAX_CHECKED; read the outcome with last_status()).
    """

    nside: int
    n_steps: int
    freq_hz: tuple
    model_id: int
    theta: np.ndarray
    r_max_kpc: float = 20.0
    obs_kpc: tuple = OBS_CONFIG_KPC
    box_clip: bool = False
    box_kpc: tuple = BOX_PAPER_KPC
    f64: bool = False
    pix_begin: int = 0
    pix_count: int = 0
    rm_rule: int = 0
    grid: np.ndarray | None = None
    checked: bool = False

    def __post_init__(self):
        self.theta = np.asarray(self.theta, dtype=np.float64).copy()
        self.freq_hz = tuple(float(f) for f in self.freq_hz)
        if self.grid is not None:
            if not hasattr(self.grid, "data_ptr"):       # host array: a private, read-only copy
                self.grid = np.array(self.grid, dtype=np.float64)
                self.grid.setflags(write=False)
            shape = tuple(self.grid.shape)
            if len(shape) != 4 or shape[3] != 3 or min(shape[:3]) < 2:
                raise ValueError("grid must be [nz][ny][nx][3] with every n >= 2")

    @property
    def npix(self) -> int:
        return 12 * self.nside * self.nside

    @property
    def n_pix_out(self) -> int:
        return self.pix_count if self.pix_count else self.npix - self.pix_begin

    @property
    def n_freq(self) -> int:
        return len(self.freq_hz)

    @property
    def samples(self) -> int:
        """LOS integration points of one map (Sec. 4.2: 12 NSIDE^2 N_int)."""
        return self.n_pix_out * self.n_steps

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    def with_theta(self, theta) -> "Problem":
        return dataclasses.replace(self, theta=np.asarray(theta, dtype=np.float64).copy())


# ---------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------
FREQS_C1 = (408e6, 1.4e9)
FREQS_C2 = (408e6, 1.4e9, 2.3e9, 23e9)


def toy_theta(Bx=6.0, By=0.0, Bz=0.0, ne=0.01, N0=4.01e-5, p=3.0, R0=4.0) -> np.ndarray:
    """Sec. 2.4 toy: uniform B = (6 uG, 0, 0), n_e = 0.01, N0 = 4.01e-5 cm^-3
    inside a 4 kpc sphere around the observer."""
    return np.array([Bx, By, Bz, ne, N0, p, R0], dtype=np.float64)


def toy_problem(nside=64, n_steps=1024, freq_hz=(2.4e9,), box_clip=True, **kw) -> Problem:
    """The paper's accuracy test (Sec. 2.4): NSIDE 64, N_int 1024, 2.4 GHz,
    box (40, 40, 10) kpc, observer at (-8.3, 0, 0.006) kpc."""
    return Problem(nside=nside, n_steps=n_steps, freq_hz=freq_hz, model_id=MODEL_TOY,
                   theta=kw.pop("theta", toy_theta()), obs_kpc=kw.pop("obs_kpc", OBS_PAPER_KPC),
                   box_clip=box_clip, **kw)


def wmap_theta() -> np.ndarray:
    """Plain-forward workload at Nside 16: b0 = 6 uG, pitch psi0 = 11.5 deg,
    psi1 = chi0B = 0, uniform 1 uG x field, N0(obs) = 4e-5 cm^-3, p = 3,
    n_e0 = 0.03 cm^-3."""
    return np.array([6.0, math.radians(11.5), 0.0, 0.0, 1.0, N0_EARTH, 3.0, 0.03])


def config1() -> Problem:
    """Nside 16, 128 steps to 20 kpc, WMAP-type field, 408 MHz and 1.4 GHz, FP64."""
    return Problem(nside=16, n_steps=128, freq_hz=FREQS_C1, model_id=MODEL_WMAP,
                   theta=wmap_theta(), f64=True)


def jf12_fiducial(seed: int = 2) -> np.ndarray:
    """JF12-type parameters: arm strengths U[-3, 3] uG and p U[2.8, 3.2] drawn
    from `seed`; halo B_h = 1.4 uG, z_h = 5.3 kpc; X field B_X = 4.6 uG,
    theta_X = 49 deg; N0(obs) = 4e-5 cm^-3; n_e scale heights 1.0 and 0.15 kpc."""
    arms = uniform(substream(seed, 1), 8, -3.0, 3.0)
    p = float(uniform(substream(seed, 2), 1, 2.8, 3.2)[0])
    return np.concatenate([arms, [1.4, 5.3, 4.6, math.radians(49.0), N0_EARTH, p, 1.0, 0.15]])


#: Scale of each JF12 parameter for relative steps: |theta_i|, 3 uG for arms.
def jf12_scales(theta) -> np.ndarray:
    s = np.abs(np.asarray(theta, dtype=np.float64)).copy()
    s[:8] = 3.0
    return s


def config2(seed: int = 2) -> Problem:
    """Nside 64, 512 steps to 20 kpc, JF12-type field, four frequencies, FP32."""
    return Problem(nside=64, n_steps=512, freq_hz=FREQS_C2, model_id=MODEL_JF12,
                   theta=jf12_fiducial(seed))


def perturbed_theta(theta, seed: int = 3, frac: float = 0.05) -> np.ndarray:
    """theta + N(0, (frac * scale_i)^2), scale = |theta_i| (3 uG for arms)."""
    theta = np.asarray(theta, dtype=np.float64)
    return theta + frac * jf12_scales(theta) * normal(substream(seed, 1), theta.size)


def target_noise(shape, seed: int = 3, sigma: float = 0.5) -> np.ndarray:
    """Gaussian map noise N(0, sigma^2) in K, for the chi^2 target."""
    n = int(np.prod(shape))
    return (sigma * normal(substream(seed, 2), n)).reshape(shape)


def config3(seed: int = 3) -> tuple[Problem, np.ndarray, float]:
    """Adjoint workload: the Nside-64 JF12-type model, its 16 parameters free.
    Returns (problem at the fiducial theta, the perturbed theta that generates
    the target map, sigma = 0.5 K).  The caller renders the target map with a
    forward model of its choice and adds target_noise()."""
    prob = config2()
    return prob, perturbed_theta(prob.theta, seed), 0.5


NSIDE_CHOICES = (16, 32, 64, 128)
STEP_CHOICES = (128, 256, 512, 1024)


def config4(n_sets: int = 256, seed: int = 4) -> list[Problem]:
    """Batched ensemble: theta ~ N(theta_fid, (0.05 |theta_fid|)^2) (arms 0.15 uG),
    p clipped to [2.8, 3.2]; Nside and steps drawn uniformly per set."""
    fid = jf12_fiducial(2)
    scale = jf12_scales(fid)
    sets = []
    g = normal(substream(seed, 1), n_sets * fid.size).reshape(n_sets, fid.size)
    u_ns = splitmix64(substream(seed, 2), n_sets)
    u_st = splitmix64(substream(seed, 3), n_sets)
    for k in range(n_sets):
        th = fid + 0.05 * scale * g[k]
        th[13] = min(max(th[13], 2.8), 3.2)
        nside = NSIDE_CHOICES[int(u_ns[k] % np.uint64(4))]
        steps = STEP_CHOICES[int(u_st[k] % np.uint64(4))]
        sets.append(Problem(nside=nside, n_steps=steps, freq_hz=FREQS_C2,
                            model_id=MODEL_JF12, theta=th))
    return sets


def config5_thetas(n: int = 50000, seed: int = 50, frac: float = 0.2) -> np.ndarray:
    """Surrogate training draws: theta ~ U[theta_fid -/+ frac * scale_i]."""
    fid = jf12_fiducial(2)
    scale = jf12_scales(fid)
    u = uniform(substream(seed, 1), n * fid.size, -1.0, 1.0).reshape(n, fid.size)
    th = fid[None, :] + frac * scale[None, :] * u
    return th


def sample_pixels(npix: int, count: int, seed: int = 11) -> np.ndarray:
    """`count` distinct pixel indices in [0, npix), sorted, from a seeded stream."""
    count = min(count, npix)
    keys = splitmix64(substream(seed, npix), npix)
    return np.sort(np.argsort(keys, kind="stable")[:count]).astype(np.int64)


# ---------------------------------------------------------------------------
# learned surrogate (parameters -> basis coefficients of a 408 MHz map)
# ---------------------------------------------------------------------------

SURROGATE_FREQ_HZ = (408e6,)
SURROGATE_WIDTHS = (16, 1024, 1024, 1024, 1024, 3 * 3072)


def config5_box(frac: float = 0.2) -> tuple[np.ndarray, np.ndarray]:
    """The training box theta_fid -/+ frac * scale_i as (lo, hi)."""
    fid = jf12_fiducial(2)
    scale = jf12_scales(fid)
    return fid - frac * scale, fid + frac * scale


def config5_problem() -> Problem:
    """The map the surrogate emulates: Nside 64, 512 steps, 408 MHz, JF12-type."""
    return config2().replace(freq_hz=SURROGATE_FREQ_HZ)


def surrogate_basis_spec(nside: int, n_basis: int, seed: int = 5) -> tuple[np.ndarray, np.ndarray]:
    """Seeded draws defining the basis: a sign per pixel (+1/-1, int8) and
    n_basis distinct row indices in [0, 12 nside^2) (int32, in draw order)."""
    npix = 12 * nside * nside
    if not 1 <= n_basis <= npix:
        raise ValueError("n_basis must be in [1, npix]")
    signs = np.where((splitmix64(substream(seed, 1), npix) >> np.uint64(63)) == 0, 1, -1).astype(np.int8)
    keys = splitmix64(substream(seed, 2), npix)
    rows = np.argsort(keys, kind="stable")[:n_basis].astype(np.int32)
    return signs, rows


def mlp_init(widths=SURROGATE_WIDTHS, seed: int = 7) -> list[tuple[np.ndarray, np.ndarray]]:
    """Initial weights: W_l ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) of shape
    [out, in] (float32), biases zero."""
    params = []
    for l in range(len(widths) - 1):
        fan_in, fan_out = widths[l], widths[l + 1]
        b = 1.0 / math.sqrt(fan_in)
        w = uniform(substream(seed, l + 1), fan_out * fan_in, -b, b).reshape(fan_out, fan_in)
        params.append((w.astype(np.float32), np.zeros(fan_out, dtype=np.float32)))
    return params


# ---------------------------------------------------------------------------
# grid model (B on a regular grid over the box, Sec. 3.3)
# ---------------------------------------------------------------------------

def grid_field(n=GRID_PAPER_N, seed: int = 21, n_modes: int = 8, amp_ug: float = 4.0) -> np.ndarray:
    """A seeded smooth vector field on an (nx, ny, nz) node lattice, returned
    as [nz][ny][nx][3] float64 (uG): a sum of n_modes plane waves over the node
    indices, B_c[k, j, i] = sum_m a_mc cos(2 pi (kx_m i / nx + ky_m j / ny +
    kz_m k / nz) + phi_m), wave numbers integers in [-3, 3], a_mc ~ N(0,
    amp^2 / n_modes), phi_m ~ U[0, 2 pi)."""
    nx, ny, nz = (int(v) for v in n)
    waves = (splitmix64(substream(seed, 1), 3 * n_modes) % np.uint64(7)).astype(np.int64).reshape(n_modes, 3) - 3
    amps = (amp_ug / math.sqrt(n_modes)) * normal(substream(seed, 2), 3 * n_modes).reshape(n_modes, 3)
    phases = uniform(substream(seed, 3), n_modes, 0.0, 2.0 * math.pi)
    i = np.arange(nx, dtype=np.float64)[None, None, :] / nx
    j = np.arange(ny, dtype=np.float64)[None, :, None] / ny
    k = np.arange(nz, dtype=np.float64)[:, None, None] / nz
    out = np.zeros((nz, ny, nx, 3), dtype=np.float64)
    for m in range(n_modes):
        wave = np.cos(2.0 * math.pi * (waves[m, 0] * i + waves[m, 1] * j + waves[m, 2] * k) + phases[m])
        out += wave[..., None] * amps[m][None, None, None, :]
    return out


def grid_theta(N0_obs: float = N0_EARTH, p: float = 3.0, ne0: float = 0.03) -> np.ndarray:
    """Grid-model parameters [N0_obs (cm^-3), p, ne0 (cm^-3)]."""
    return np.array([N0_obs, p, ne0], dtype=np.float64)


def grid_problem(nside: int = 64, n_steps: int = 512, freq_hz=(2.4e9,), n=GRID_PAPER_N, seed: int = 21,
                 **kw) -> Problem:
    """The grid optimisation workload (Sec. 3.3): Nside 64, 512 steps to the
    walls of the (40, 40, 10) kpc box, Q/U at 2.4 GHz, B on 128 x 128 x 32
    nodes (grid_field(seed)), analytic CR and thermal electrons."""
    return Problem(nside=nside, n_steps=n_steps, freq_hz=freq_hz, model_id=MODEL_GRID,
                   theta=kw.pop("theta", grid_theta()), box_clip=True, grid=kw.pop("grid", grid_field(n, seed)),
                   **kw)


# ---------------------------------------------------------------------------
# stacked WMAP model (Sec. 4.3, Eq. 16)
# ---------------------------------------------------------------------------

#: b0 (uG), psi0, psi1, chi0B (rad) of the four WMAP fields (Sec. 4.3, table of model parameters).
WMAP_STACK_TABLE = ((1.20, 0.4712, 0.0157, 0.4363),
                    (3.50, 0.6457, 0.5393, 0.6108),
                    (7.70, 1.1693, 1.0629, 1.1344),
                    (5.70, 1.6930, 1.5865, 1.6580))


def wmap_stack_theta(N0_obs: float = N0_EARTH, p: float = 3.0, ne0: float = 0.03) -> np.ndarray:
    """The 16 field parameters of Sec. 4.3's table, then N0_obs, p, ne0."""
    return np.array([v for row in WMAP_STACK_TABLE for v in row] + [N0_obs, p, ne0], dtype=np.float64)


def wmap_stack_problem(nside: int = 64, n_steps: int = 512, freq_hz=(2.4e9,), **kw) -> Problem:
    """Sec. 4.3's workload: the stacked model in the (40, 40, 10) kpc box,
    Nside 64, 512 steps, Q/U at 2.4 GHz, observer as in Sec. 2.1."""
    return Problem(nside=nside, n_steps=n_steps, freq_hz=freq_hz, model_id=MODEL_WMAP_STACK,
                   theta=kw.pop("theta", wmap_stack_theta()), box_clip=kw.pop("box_clip", True),
                   obs_kpc=kw.pop("obs_kpc", OBS_PAPER_KPC), **kw)
