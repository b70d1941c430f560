"""Pins of the oracle's WMAP-type field (Sec. 3.1: the direction of Eq. 13
under an exponential envelope of this project's, plus a uniform x field)
by properties its definition implies, not by its formula retyped:

W1 with the x field off, the direction at every point is Eq. 13's: the
   elevation out of the plane is chi = chi0B tanh(z / 1 kpc) and the
   horizontal part makes the pitch angle psi = psi0 + psi1 ln(rho / 8 kpc)
   from rho^ towards phi^ inside 3 <= rho <= 20 kpc; outside, B is along rho^;
W2 |B| depends on rho and |z| only (axisymmetric, even in z);
W3 the x field adds exactly (B_ux, 0, 0) everywhere (superposition);
W4 N0 at the observer is N0_obs, n_e at the Galactic centre is n_e0, and
   the I map falls as nu^{-(p+3)/2} with p = theta[6] (I carries no
   Faraday rotation).
The envelope's absolute values are this project's choice and are not pinned.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2410_01136_gb300 import inputs as I


def problem(psi0=0.35, psi1=0.4, chi0=0.6, bux=0.0, **kw):
    th = I.wmap_theta()
    th[1], th[2], th[3], th[4] = psi0, psi1, chi0, bux
    return I.Problem(nside=kw.get("nside", 1), n_steps=kw.get("n_steps", 4), freq_hz=kw.get("freq_hz", (1.4e9,)),
                     model_id=I.MODEL_WMAP, theta=th)


def points(n=400, seed=70):
    u = I.uniform(I.substream(seed, 1), 3 * n, 0.0, 1.0).reshape(n, 3)
    rho = 0.5 + 24.5 * u[:, 0]
    phi = 2 * math.pi * u[:, 1]
    z = -4.0 + 8.0 * u[:, 2]
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def test_w1_direction():
    prob = problem()
    _, psi0, psi1, chi0 = prob.theta[:4]
    B = oracle.fields_batch(prob, points(), np.zeros(400))[:, :3]
    n_in = 0
    for r, b in zip(points(), B):
        rho = math.hypot(r[0], r[1])
        rh = np.array([r[0] / rho, r[1] / rho, 0.0])
        ph = np.array([-r[1] / rho, r[0] / rho, 0.0])
        mag = np.linalg.norm(b)
        if 3.0 <= rho <= 20.0:
            n_in += 1
            chi = chi0 * math.tanh(r[2])
            assert b[2] / mag == pytest.approx(math.sin(chi), abs=1e-12)
            ang = math.atan2(b @ ph, b @ rh)
            psi = psi0 + psi1 * math.log(rho / 8.0)
            assert math.remainder(ang - psi, 2 * math.pi) == pytest.approx(0.0, abs=1e-9)
        else:
            np.testing.assert_allclose(b / mag, rh, rtol=0, atol=1e-12)
    assert n_in > 200


def test_w2_axisymmetric_and_even():
    prob = problem()
    r = points(200, seed=71)
    mag = np.linalg.norm(oracle.fields_batch(prob, r, np.zeros(200))[:, :3], axis=1)
    rot = np.stack([-r[:, 1], r[:, 0], -r[:, 2]], axis=1)        # phi + 90 deg, z -> -z
    mag2 = np.linalg.norm(oracle.fields_batch(prob, rot, np.zeros(200))[:, :3], axis=1)
    np.testing.assert_allclose(mag2, mag, rtol=1e-13)


def test_w3_uniform_x_field():
    r = points(200, seed=72)
    a = oracle.fields_batch(problem(bux=0.0), r, np.zeros(200))[:, :3]
    b = oracle.fields_batch(problem(bux=1.7), r, np.zeros(200))[:, :3]
    np.testing.assert_allclose(b - a, np.tile([1.7, 0.0, 0.0], (200, 1)), rtol=0, atol=1e-13)


def test_w4_densities_and_index():
    prob = problem(nside=2, n_steps=64, freq_hz=(1.0e9, 4.0e9))
    th = prob.theta.copy()
    th[5], th[6], th[7] = 3.1e-5, 2.6, 0.045
    prob = prob.with_theta(th)
    _, n0, _ = oracle.fields(prob, prob.obs_kpc)
    assert n0 == pytest.approx(3.1e-5, rel=1e-12)
    _, _, ne = oracle.fields(prob, (0.0, 0.0, 0.0))
    assert ne == pytest.approx(0.045, rel=1e-12)
    m = oracle.forward(prob)
    np.testing.assert_allclose(m[0, 0] / m[1, 0], 4.0 ** ((2.6 + 3) / 2), rtol=1e-10)
