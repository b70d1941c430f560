"""Pins of the oracle's stacked WMAP model (Sec. 4.3, Eq. 16; components of
the form of Eq. 13) against properties of its definition that do not come
from the oracle's code.

S1  one component alone: |B| = w_k b0_k everywhere (each Eq. 13 field has
    constant magnitude b0; weights 0.6, 0.3, 0.1, 0.3)
S2  one component alone, mapped back through its permutation of Eq. 16:
    the elevation is chi = chi0B tanh(z / 1 kpc) and the pitch angle from
    rho^ towards phi^ is psi = psi0 + psi1 ln(rho / 8 kpc) inside
    3 <= rho <= 20 kpc, and the field is b0 rho^ outside (this fixes each
    component's permutation and weight)
S3  superposition: the stacked field is the sum of its single-component fields
S4  N0 at the observer is N0_obs, n_e at the Galactic centre is n_e0, and
    without Faraday rotation the I map falls as nu^{-(p+3)/2} (theta[17] is p)
"""
import math

import numpy as np
import pytest

import oracle
from paper_2410_01136_gb300 import inputs as I

WEIGHTS = (0.6, 0.3, 0.1, 0.3)
# component k's (x, y, z) -> position in the stacked (x, y, z) of Eq. 16
PERM = ((0, 1, 2), (0, 2, 1), (2, 1, 0), (1, 0, 2))


def single(k, theta=None):
    th = I.wmap_stack_theta() if theta is None else np.array(theta, dtype=float)
    for j in range(4):
        if j != k:
            th[4 * j] = 0.0
    return I.wmap_stack_problem(nside=1, n_steps=4, theta=th)


def points(n=400, seed=60):
    u = I.uniform(I.substream(seed, 1), 3 * n, -0.5, 0.5).reshape(n, 3)
    return u * np.array(I.BOX_PAPER_KPC)


def back(k, B):
    """Component k's own (x, y, z) from its contribution to the stacked field."""
    v = np.empty(3)
    for a in range(3):
        v[a] = B[PERM[k][a]]
    return v / WEIGHTS[k]


@pytest.mark.parametrize("k", range(4))
def test_s1_magnitude(k):
    prob = single(k)
    b0 = prob.theta[4 * k]
    for r in points():
        B, _, _ = oracle.fields(prob, r)
        assert np.linalg.norm(B) == pytest.approx(WEIGHTS[k] * b0, rel=1e-12)


@pytest.mark.parametrize("k", range(4))
def test_s2_pitch_and_elevation(k):
    prob = single(k)
    b0, psi0, psi1, chi0 = prob.theta[4 * k:4 * k + 4]
    n_in = 0
    for r in points(seed=61):
        B, _, _ = oracle.fields(prob, r)
        v = back(k, B)
        rho = math.hypot(r[0], r[1])
        rh = np.array([r[0] / rho, r[1] / rho, 0.0])
        ph = np.array([-r[1] / rho, r[0] / rho, 0.0])
        if 3.0 <= rho <= 20.0:
            n_in += 1
            chi = chi0 * math.tanh(r[2])
            assert v[2] == pytest.approx(b0 * math.sin(chi), abs=1e-12 * b0)
            psi = psi0 + psi1 * math.log(rho / 8.0)
            # the horizontal part is b0 cos(chi) (cos psi, sin psi): its sign
            # flips where |chi| > pi/2 (model 4 has chi0B = 1.658)
            cc = math.cos(chi)
            if abs(cc) > 1e-6:
                ang = math.atan2((v @ ph) / cc, (v @ rh) / cc)
                assert math.remainder(ang - psi, 2 * math.pi) == pytest.approx(0.0, abs=1e-9)
        else:
            np.testing.assert_allclose(v, b0 * rh, rtol=0, atol=1e-12 * b0)
    assert n_in > 100


def test_s3_superposition():
    full = I.wmap_stack_problem(nside=1, n_steps=4)
    for r in points(50, seed=62):
        B, _, _ = oracle.fields(full, r)
        parts = sum(oracle.fields(single(k), r)[0] for k in range(4))
        np.testing.assert_allclose(B, parts, rtol=0, atol=1e-12)


def test_s4_n0_ne_and_p():
    th = I.wmap_stack_theta(N0_obs=3.3e-5, p=2.7, ne0=0.041)
    prob = I.wmap_stack_problem(nside=2, n_steps=64, theta=th, freq_hz=(1.0e9, 4.0e9))
    _, n0, _ = oracle.fields(prob, prob.obs_kpc)
    assert n0 == pytest.approx(3.3e-5, rel=1e-12)
    _, _, ne = oracle.fields(prob, (0.0, 0.0, 0.0))
    assert ne == pytest.approx(0.041, rel=1e-12)
    m = oracle.forward(prob)
    ratio = m[0, 0] / m[1, 0]
    np.testing.assert_allclose(ratio, 4.0 ** ((2.7 + 3) / 2), rtol=1e-10)
