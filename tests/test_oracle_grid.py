"""Pins of the oracle's grid model (B on a regular grid over the box, found
at the midpoints by 3D linear interpolation; Sec. 2.3, Sec. 3.3) against
facts that do not come from the oracle itself.

G1  trilinear interpolation reproduces any field that is linear in each
    coordinate separately (a + b x + c y + d z + cross terms up to x y z)
    sampled at the nodes, everywhere inside the box: this fixes where the
    nodes sit (wall to wall), the axis order and the [nz][ny][nx][3] layout
G2  a random grid agrees with scipy's RegularGridInterpolator (linear) over
    the same wall-to-wall node coordinates
G3  node values come back exactly at node positions
G4  beyond a wall the field keeps the wall's value (the clamp)
G5  a uniform grid field marches to the same maps as the WMAP-type model
    with b0 = 0 and the same uniform x field, so the grid model's CR density,
    n_e and spectral index are the WMAP-type model's
G6  the model evaluation (oracle.fields) returns the interpolated B
"""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle
from paper_2410_01136_gb300 import inputs as I

BOX = I.BOX_PAPER_KPC


def _nodes(n, l):
    return np.linspace(-0.5 * l, 0.5 * l, n)


def _sample(fn, n=(9, 7, 5), box=BOX):
    """Grid [nz][ny][nx][3] of fn(x, y, z) -> 3-vector at wall-to-wall nodes."""
    x, y, z = (_nodes(n[a], box[a]) for a in range(3))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack(fn(X, Y, Z), axis=-1)


def _points(count, seed, box=BOX, pad=0.0):
    u = I.uniform(I.substream(seed, 1), 3 * count, -0.5, 0.5).reshape(count, 3)
    return u * (np.asarray(box) * (1.0 + pad))


def _multilinear(X, Y, Z):
    return (1.5 + 0.3 * X - 0.2 * Y + 0.7 * Z + 0.01 * X * Y - 0.05 * Y * Z + 0.002 * X * Y * Z,
            -2.0 + 0.1 * X + 0.4 * Y - 0.3 * Z + 0.02 * X * Z,
            0.25 - 0.15 * X + 0.05 * Y + 1.1 * Z - 0.003 * X * Y * Z)


def test_g1_multilinear_exact():
    grid = _sample(_multilinear)
    for r in _points(200, seed=31):
        want = np.array(_multilinear(*r))
        got = oracle.grid_interp(grid, BOX, r)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_g1_detects_cell_centred_nodes():
    """The same linear field sampled at cell centres is NOT reproduced: the
    pin distinguishes the two node conventions."""
    n = (9, 7, 5)
    x, y, z = ((np.arange(n[a]) + 0.5) * BOX[a] / n[a] - 0.5 * BOX[a] for a in range(3))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    grid = np.stack(_multilinear(X, Y, Z), axis=-1)
    r = np.array([3.1, -2.2, 1.3])
    assert np.max(np.abs(oracle.grid_interp(grid, BOX, r) - np.array(_multilinear(*r)))) > 1e-3


def test_g2_matches_scipy():
    n = (11, 6, 4)
    g = I.normal(I.substream(32, 1), n[2] * n[1] * n[0] * 3).reshape(n[2], n[1], n[0], 3)
    axes = (_nodes(n[2], BOX[2]), _nodes(n[1], BOX[1]), _nodes(n[0], BOX[0]))
    pts = _points(300, seed=33)
    for c in range(3):
        rgi = RegularGridInterpolator(axes, g[..., c], method="linear")
        want = rgi(pts[:, ::-1])
        got = np.array([oracle.grid_interp(g, BOX, r)[c] for r in pts])
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_g3_nodes_exact():
    n = (5, 4, 3)
    g = I.normal(I.substream(34, 1), n[2] * n[1] * n[0] * 3).reshape(n[2], n[1], n[0], 3)
    x, y, z = (_nodes(n[a], BOX[a]) for a in range(3))
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                got = oracle.grid_interp(g, BOX, (x[i], y[j], z[k]))
                np.testing.assert_allclose(got, g[k, j, i], rtol=0, atol=1e-13)


def test_g4_clamp_beyond_walls():
    grid = _sample(_multilinear)
    r_in = np.array([20.0, -20.0, 5.0])        # corner of the box
    r_out = np.array([25.0, -31.0, 9.0])       # beyond it on all three axes
    want = np.array(_multilinear(*r_in))
    np.testing.assert_allclose(oracle.grid_interp(grid, BOX, r_in), want, atol=1e-12)
    np.testing.assert_allclose(oracle.grid_interp(grid, BOX, r_out), want, atol=1e-12)
    # beyond one wall only: the other coordinates still interpolate
    r = np.array([3.0, 1.0, 7.5])
    np.testing.assert_allclose(oracle.grid_interp(grid, BOX, r),
                               np.array(_multilinear(3.0, 1.0, 5.0)), atol=1e-12)


def test_g5_uniform_grid_equals_wmap_model():
    bux = 2.5
    grid = _sample(lambda X, Y, Z: (bux + 0 * X, 0 * Y, 0 * Z), n=(4, 3, 2))
    th = I.grid_theta(N0_obs=4.1e-5, p=2.9, ne0=0.04)
    pg = I.Problem(nside=2, n_steps=64, freq_hz=(408e6, 2.4e9), model_id=I.MODEL_GRID, theta=th,
                   box_clip=True, grid=grid)
    wm = np.array([0.0, 0.3, 0.0, 0.0, bux, th[0], th[1], th[2]])
    pw = I.Problem(nside=2, n_steps=64, freq_hz=(408e6, 2.4e9), model_id=I.MODEL_WMAP, theta=wm,
                   box_clip=True)
    mg = oracle.forward(pg)
    mw = oracle.forward(pw)
    assert np.all(np.isfinite(mg)) and np.abs(mg).max() > 0
    np.testing.assert_allclose(mg, mw, rtol=1e-11, atol=1e-18)   # weights sum to 1 up to rounding


def test_g6_fields_use_the_grid():
    grid = I.grid_field(n=(6, 5, 4), seed=35)
    prob = I.Problem(nside=2, n_steps=8, freq_hz=(2.4e9,), model_id=I.MODEL_GRID, theta=I.grid_theta(),
                     box_clip=True, grid=grid)
    for r in _points(20, seed=36):
        B, n0, ne = oracle.fields(prob, r)
        np.testing.assert_allclose(B, oracle.grid_interp(grid, BOX, r), rtol=0, atol=1e-13)
        assert n0 > 0 and ne > 0


def test_grid_model_needs_box_and_grid():
    grid = I.grid_field(n=(3, 3, 2), seed=37)
    prob = I.Problem(nside=1, n_steps=4, freq_hz=(2.4e9,), model_id=I.MODEL_GRID, theta=I.grid_theta(),
                     box_clip=False, grid=grid)
    with pytest.raises(Exception):
        oracle.forward(prob)
    with pytest.raises(ValueError):
        I.Problem(nside=1, n_steps=4, freq_hz=(2.4e9,), model_id=I.MODEL_GRID, theta=I.grid_theta(),
                  box_clip=True, grid=np.zeros((1, 3, 3, 3)))


def test_grid_field_recipe_is_seeded():
    a = I.grid_field(n=(8, 6, 4), seed=21)
    b = I.grid_field(n=(8, 6, 4), seed=21)
    c = I.grid_field(n=(8, 6, 4), seed=22)
    assert a.shape == (4, 6, 8, 3)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_g7_one_ulp_response_is_a_linear_conditioning_measure():
    """The FP32 floor of the grid tests (tests/parity.py) is the oracle's
    response to moving every grid value by one float32 ulp.  Pinned here as a
    first-order (linear) response: two ulps in the same directions move
    Q + iU twice as far (to 10 %), the response is far below the unrotated
    polarised intensity P0 = Pi I (Pi = (p+1)/(p+7/3), the polarised fraction
    of Eq. 2 and 5; below 1e-4 P0) on every pixel, and at 2.4 GHz (the grid workload's
    frequency) 16 times the response stays below 1e-4 |P| on every pixel, so
    the floor acts only where the Faraday rotation depolarises."""
    import oracle
    from paper_2410_01136_gb300 import inputs
    from tests.parity import ulp_perturbed_grid
    oracle.build()
    prob = inputs.grid_problem(nside=4, n_steps=48, freq_hz=(408e6, 2.4e9), n=(12, 10, 6))
    prob = prob.replace(grid=np.asarray(prob.grid, dtype=np.float32).astype(np.float64))
    ref = oracle.forward(prob)
    P = ref[:, 1] + 1j * ref[:, 2]
    d1 = oracle.forward(prob.replace(grid=ulp_perturbed_grid(prob.grid, 5, 1)))
    d2 = oracle.forward(prob.replace(grid=ulp_perturbed_grid(prob.grid, 5, 2)))
    r1 = (d1[:, 1] + 1j * d1[:, 2]) - P
    r2 = (d2[:, 1] + 1j * d2[:, 2]) - P
    big = np.abs(r1) > 1e-3 * np.abs(r1).max()
    np.testing.assert_allclose(r2[big], 2 * r1[big], rtol=0.1, atol=0)
    p = prob.theta[1]
    P0 = (p + 1) / (p + 7 / 3) * ref[:, 0]
    assert np.all(np.abs(r1) <= 1e-4 * P0)
    den = np.maximum(np.abs(P[1]), 1e-2 * np.median(np.abs(P[1])))
    assert np.all(16 * np.abs(r1[1]) < 1e-4 * den)
