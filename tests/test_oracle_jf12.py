"""Pins of the oracle's JF12-type field (the model this project defines after
Jansson & Farrar 2012 for the 16-parameter workload; the paper cites that
field without printing it).  Each pin is a property the definition implies,
not its formula retyped, chosen so that a plausible slip fails one of them:

J1 the spiral disc is divergence-free wherever its radial window is flat, at
   any height (fixes the pitch and its sign in the arm coordinate against
   the field's direction, and the 1/rho scaling);
J2 the disc field's pitch angle is 11.5 deg (B_rho / B_phi = tan i), so the
   cylindrical-to-Cartesian rotation is not transposed;
J3 with equal arm strengths |B| rho does not depend on rho or phi (the arm
   weights are a partition of unity);
J4 along a circle, arm strengths that alternate high and low are met as 8
   extrema in the cyclic order b_1..b_8 of increasing phi (arm count, layout
   and winding);
J5 the halo is purely azimuthal, divergence-free and odd in z;
J6 the X field is poloidal; away from the plane its field lines keep
   r_p = rho - |z| / tan theta_X and it is divergence-free up to the smooth
   sign's departure from +-1; it vanishes where r_p <= 0;
J7 n_e at the Galactic centre is 0.025 + 0.10 cm^-3, N0 at the observer is
   N0_obs."""
import math

import numpy as np
import pytest

from paper_2410_01136_gb300 import inputs

oracle = pytest.importorskip("oracle")


@pytest.fixture(scope="module")
def base():
    oracle.build()
    return inputs.config2()


def with_parts(prob, disc=True, halo=True, xfield=True, arms=None):
    th = prob.theta.copy()
    if arms is not None:
        th[:8] = arms
    if not disc:
        th[:8] = 0.0
    if not halo:
        th[8] = 0.0
    if not xfield:
        th[10] = 0.0
    return prob.with_theta(th)


def B_at(prob, r):
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    return oracle.fields_batch(prob, r, np.zeros(len(r)))[:, :3]


def divergence(prob, r, h=1e-4):
    r = np.atleast_2d(r)
    div = np.zeros(len(r))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        div += (B_at(prob, r + e)[:, k] - B_at(prob, r - e)[:, k]) / (2 * h)
    return div


def cyl_points(n, rho_lo, rho_hi, z_lo, z_hi, seed):
    u = np.random.default_rng(seed).random((n, 3))
    rho = rho_lo + (rho_hi - rho_lo) * u[:, 0]
    phi = 2 * np.pi * u[:, 1]
    z = z_lo + (z_hi - z_lo) * u[:, 2]
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def cyl_components(r, B):
    rho = np.hypot(r[:, 0], r[:, 1])
    c, s = r[:, 0] / rho, r[:, 1] / rho
    return B[:, 0] * c + B[:, 1] * s, -B[:, 0] * s + B[:, 1] * c, B[:, 2]


def test_j1_disc_divergence_free(base):
    prob = with_parts(base, halo=False, xfield=False)
    r = cyl_points(400, 5.3, 19.7, -2.0, 2.0, seed=1)
    B = B_at(prob, r)
    scale = np.abs(B).max()
    assert scale > 0.1
    assert np.abs(divergence(prob, r)).max() < 1e-6 * scale


def test_j1_divergence_test_is_sensitive(base):
    """The same check fails for a field with a different pitch in its
    direction than in its spiral (what a pitch slip would give)."""
    prob = with_parts(base, halo=False, xfield=False)
    r = cyl_points(50, 6.0, 18.0, -0.5, 0.5, seed=2)

    def tilted(rr):
        B = B_at(prob, rr)
        rho = np.hypot(rr[:, 0], rr[:, 1])
        c, s = rr[:, 0] / rho, rr[:, 1] / rho
        br, bp, bz = cyl_components(rr, B)
        br = 1.2 * br                                   # pitch no longer 11.5 deg
        return np.stack([br * c - bp * s, br * s + bp * c, bz], axis=1)

    h = 1e-4
    div = np.zeros(len(r))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        div += (tilted(r + e)[:, k] - tilted(r - e)[:, k]) / (2 * h)
    assert np.abs(div).max() > 1e-3 * np.abs(B_at(prob, r)).max()


def test_j2_disc_pitch(base):
    prob = with_parts(base, halo=False, xfield=False)
    r = cyl_points(300, 3.0, 22.0, -3.0, 3.0, seed=3)
    B = B_at(prob, r)
    br, bp, bz = cyl_components(r, B)
    live = np.abs(bp) > 1e-9
    assert live.sum() > 200
    assert np.allclose(br[live] / bp[live], math.tan(math.radians(11.5)), rtol=1e-12)
    assert np.abs(bz).max() == 0.0


def test_j3_equal_arms_partition_of_unity(base):
    prob = with_parts(base, halo=False, xfield=False, arms=np.full(8, 2.0))
    for z in (0.0, 0.7, -1.3):
        r = cyl_points(300, 5.3, 19.7, z, z, seed=4)
        rho = np.hypot(r[:, 0], r[:, 1])
        g = np.linalg.norm(B_at(prob, r), axis=1) * rho
        assert np.ptp(g) < 1e-12 * g.max()


def test_j4_arm_layout_and_winding(base):
    b = np.array([3.0, -1.0, 2.5, -2.0, 1.5, -0.5, 2.0, -1.5])
    prob = with_parts(base, halo=False, xfield=False, arms=b)
    ones = with_parts(base, halo=False, xfield=False, arms=np.ones(8))
    phi = np.linspace(0.0, 2 * np.pi, 8000, endpoint=False)
    rho, z = 9.0, 0.3
    r = np.stack([rho * np.cos(phi), rho * np.sin(phi), np.full_like(phi, z)], axis=1)
    # signed strength beta(phi): the disc field over the equal-strength field
    br, bp, _ = cyl_components(r, B_at(prob, r))
    _, bp1, _ = cyl_components(r, B_at(ones, r))
    beta = bp / bp1
    prev, nxt = np.roll(beta, 1), np.roll(beta, -1)
    ext = np.where(((beta > prev) & (beta >= nxt)) | ((beta < prev) & (beta <= nxt)))[0]
    assert len(ext) == 8, ext
    vals = beta[ext]
    assert np.allclose(np.sort(vals), np.sort(b), atol=1e-5)
    # in order of increasing phi the extrema run through b_1..b_8 cyclically
    start = int(np.argmin(np.abs(b - vals[0])))
    assert np.allclose(vals, np.roll(b, -start), atol=1e-5)


def test_j5_halo_toroidal_divergence_free_odd(base):
    prob = with_parts(base, disc=False, xfield=False)
    r = cyl_points(300, 0.5, 25.0, -6.0, 6.0, seed=5)
    B = B_at(prob, r)
    br, bp, bz = cyl_components(r, B)
    assert np.abs(br).max() < 1e-13 * np.abs(bp).max() and np.abs(bz).max() == 0.0
    assert np.abs(divergence(prob, r)).max() < 1e-7 * np.abs(B).max()
    flip = r * np.array([1.0, 1.0, -1.0])
    assert np.allclose(B_at(prob, flip), -B, rtol=0, atol=1e-14 * np.abs(B).max())


def test_j6_x_field_lines_and_flux(base):
    prob = with_parts(base, disc=False, halo=False)
    thx = base.theta[11]
    # poloidal everywhere
    r = cyl_points(300, 0.5, 25.0, -6.0, 6.0, seed=6)
    B = B_at(prob, r)
    br, bp, bz = cyl_components(r, B)
    assert np.abs(bp).max() < 1e-13 * np.abs(B).max()
    # away from the plane (|s(z)| within 6e-4 of 1): lines of constant r_p
    # and nearly zero divergence; a missing r_p/rho factor or a wrong cone
    # gives O(1) divergence
    for zs in (1.0, -1.0):
        rr = cyl_points(300, 5.0, 20.0, 3.0 * zs, 5.0 * zs, seed=7)
        rho = np.hypot(rr[:, 0], rr[:, 1])
        live = rho - np.abs(rr[:, 2]) / math.tan(thx) > 0.05
        rr = rr[live]
        BB = B_at(prob, rr)
        br, _, bz = cyl_components(rr, BB)
        # tangent of constant r_p: d rho / d|z| = 1 / tan theta_X
        assert np.allclose(np.abs(br) / np.abs(bz), 1.0 / math.tan(thx), rtol=1e-3)
        assert np.all(np.sign(br) == zs)
        assert np.abs(divergence(prob, rr)).max() < 2e-3 * np.abs(BB).max()
    # zero inside the cone r_p <= 0
    r = cyl_points(300, 0.2, 5.0, 5.0, 8.0, seed=8)
    inside = np.hypot(r[:, 0], r[:, 1]) - np.abs(r[:, 2]) / math.tan(thx) <= 0
    assert inside.sum() > 50
    assert np.abs(B_at(prob, r[inside])).max() == 0.0


def test_j7_densities(base):
    out = oracle.fields_batch(base, np.array([[0.0, 0.0, 0.0], list(base.obs_kpc)]), np.zeros(2))
    assert out[0, 4] == pytest.approx(0.125, rel=1e-15)
    assert out[1, 3] == pytest.approx(base.theta[12], rel=1e-14)
