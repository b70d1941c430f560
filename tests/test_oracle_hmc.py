"""Pins of the HMC oracle (oracle/hmc.py) and of the host-side effective
sample size, against facts independent of their code.

H1  its momenta are the even outputs of the seeded Box-Muller stream
    (paper_2410_01136_gb300.inputs.normal), at the documented counters
H2  on a correlated 2-D Gaussian exp(-x^T A x / 2) its draws have mean 0 and
    covariance A^-1 (Monte Carlo error), so leapfrog, Hamiltonian and
    Metropolis step are right (a wrong sign, a dropped half step or a wrong
    kinetic energy biases the covariance)
H3  small steps conserve H: acceptance -> 1 as eps -> 0, with 1 - acceptance
    falling like eps^2 or faster
H4  a parameter with inverse mass 0 never moves; a prior box is never left
E1  the effective sample size of AR(1) chains with coefficient phi is
    m n (1 - phi) / (1 + phi) (the integrated autocorrelation time of AR(1))
"""
import numpy as np
import pytest

from oracle import hmc as ohmc
from paper_2410_01136_gb300 import effective_sample_size, inputs

A = np.array([[2.0, 0.8], [0.8, 1.0]])


def gauss(theta):
    return np.einsum("ci,ij,cj->c", theta, A, theta), 2.0 * theta @ A


def test_h1_momenta_are_the_seeded_normals():
    C, T, t = 3, 5, 2
    z = ohmc.momentum_normals(17, t, C, T)
    ref = inputs.normal(17, 2 * (t + 1) * C * T)[0::2][t * C * T:]
    np.testing.assert_array_equal(z.ravel(), ref)


def test_h2_gaussian_moments():
    C = 256
    draws, acc = ohmc.hmc_iterations(np.zeros((C, 2)), gauss, 120, eps=0.35, L=6, seed=5, inv_mass=[1.0, 1.0])
    x = draws[20:].reshape(-1, 2)
    assert 0.6 < acc.mean() < 1.0
    cov = np.cov(x.T)
    np.testing.assert_allclose(cov, np.linalg.inv(A), atol=0.05)
    np.testing.assert_allclose(x.mean(axis=0), 0.0, atol=0.03)


def test_h3_energy_conservation():
    rej = []
    for eps in (0.2, 0.1, 0.05):
        _, acc = ohmc.hmc_iterations(np.full((512, 2), 0.3), gauss, 4, eps=eps, L=int(round(1.0 / eps)), seed=6,
                                     inv_mass=[1.0, 1.0])
        rej.append(1.0 - acc.mean())
    assert rej[2] < 0.02 and rej[1] <= rej[0] and rej[2] <= rej[1]


def test_h4_fixed_parameter_and_box():
    draws, _ = ohmc.hmc_iterations(np.full((64, 2), [0.1, 0.7]), gauss, 30, eps=0.3, L=5, seed=7,
                                   inv_mass=[1.0, 0.0])
    assert np.all(draws[:, :, 1] == 0.7)
    draws, _ = ohmc.hmc_iterations(np.zeros((64, 2)), gauss, 30, eps=0.3, L=5, seed=8, inv_mass=[1.0, 1.0],
                                   lo=[-0.2, -5.0], hi=[0.3, 5.0])
    assert draws[:, :, 0].min() >= -0.2 and draws[:, :, 0].max() <= 0.3


@pytest.mark.parametrize("phi", [0.0, 0.5, 0.9])
def test_e1_ess_of_ar1(phi):
    n, m = 4000, 8
    e = inputs.normal(inputs.substream(9, int(phi * 10)), n * m).reshape(n, m)
    x = np.empty((n, m))
    x[0] = e[0] / np.sqrt(1 - phi ** 2)
    for i in range(1, n):
        x[i] = phi * x[i - 1] + e[i]
    ess = effective_sample_size(x[:, :, None])[0]
    want = m * n * (1 - phi) / (1 + phi)
    assert ess == pytest.approx(want, rel=0.15)
