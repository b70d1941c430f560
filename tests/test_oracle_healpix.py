"""Pins of the oracle's HEALPix RING pixel centres (Gorski et al. 2005).

healpy is not available, so the centres are checked by properties that any
correct RING pixelisation has: ring structure and counts, the Nside-1 base
pixels listed by hand, north-south mirror symmetry, vanishing vector sum,
distinctness, and an independent inverse map (ang2pix, written below from
the published RING algorithm) whose cells must be equal-area and must map
every centre back to its own index.
"""
import math

import numpy as np
import pytest


def centres(oracle, nside):
    npix = 12 * nside * nside
    zp = np.array([oracle.healpix_centre(nside, p) for p in range(npix)])
    return zp[:, 0], zp[:, 1]


def ang2pix_ring(nside, z, phi):
    """RING index of the pixel containing (z, phi), from the inverse algorithm
    of Gorski et al. 2005 (equatorial belt: two families of edge lines;
    polar caps: ring from sqrt(3(1-|z|)))."""
    N = nside
    za = abs(z)
    tt = (phi % (2 * math.pi)) / (math.pi / 2)  # in [0, 4)
    if za <= 2.0 / 3.0:
        t1 = N * (0.5 + tt)
        t2 = N * z * 0.75
        jp = int(math.floor(t1 - t2))
        jm = int(math.floor(t1 + t2))
        ir = N + 1 + jp - jm              # ring counted from z = 2/3, 1..2N+1
        kshift = 1 - (ir & 1)
        ip = (jp + jm - N + kshift + 1) // 2
        ip %= 4 * N
        return 2 * N * (N - 1) + (ir - 1) * 4 * N + ip
    tp = tt - math.floor(tt)
    tmp = N * math.sqrt(3.0 * (1.0 - za))
    jp = int(math.floor(tp * tmp))
    jm = int(math.floor((1.0 - tp) * tmp))
    ir = jp + jm + 1                      # ring counted from the nearest pole
    ip = int(math.floor(tt * ir)) % (4 * ir)
    if z > 0:
        return 2 * ir * (ir - 1) + ip
    return 12 * N * N - 2 * ir * (ir + 1) + ip


def test_nside1_base_pixels(oracle_lib):
    z, phi = centres(oracle_lib, 1)
    q = math.pi / 4
    want = [(2 / 3, q), (2 / 3, 3 * q), (2 / 3, 5 * q), (2 / 3, 7 * q),
            (0.0, 0.0), (0.0, 2 * q), (0.0, 4 * q), (0.0, 6 * q),
            (-2 / 3, q), (-2 / 3, 3 * q), (-2 / 3, 5 * q), (-2 / 3, 7 * q)]
    for p, (zw, pw) in enumerate(want):
        assert z[p] == pytest.approx(zw, abs=1e-15)
        assert phi[p] == pytest.approx(pw, abs=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 3, 4, 8])
def test_ring_structure(oracle_lib, nside):
    z, phi = centres(oracle_lib, nside)
    rings, counts = np.unique(np.round(z, 12), return_counts=True)
    assert len(rings) == 4 * nside - 1
    # rings come out north to south; counts 4, 8, ..., 4N ... 4N, ..., 8, 4
    order = np.argsort(-rings)
    c = counts[order]
    want = [4 * min(i, nside, 4 * nside - i) for i in range(1, 4 * nside)]
    assert list(c) == want
    # z is non-increasing with the pixel index, and phi increases within a ring
    assert np.all(np.diff(z) <= 1e-15)
    for r in rings:
        sel = np.where(np.round(z, 12) == r)[0]
        assert np.all(np.diff(phi[sel]) > 0)
        d = np.diff(phi[sel])
        assert np.allclose(d, 2 * math.pi / sel.size, atol=1e-13)


@pytest.mark.parametrize("nside", [1, 2, 3, 4])
def test_mirror_sum_distinct(oracle_lib, nside):
    z, phi = centres(oracle_lib, nside)
    npix = z.size
    assert np.allclose(z, -z[::-1], atol=1e-15)
    # each ring and its mirror carry the same set of azimuths
    for r in np.unique(np.round(z, 12)):
        a = np.sort(phi[np.round(z, 12) == r])
        b = np.sort(phi[np.round(z, 12) == -r]) if r != 0 else a
        assert np.allclose(a, b, atol=1e-13)
    s = np.sqrt(1 - z * z)
    v = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
    assert np.allclose(v.sum(axis=0), 0.0, atol=1e-12)
    key = {(round(a, 12), round(b, 12)) for a, b in zip(z, phi)}
    assert len(key) == npix


@pytest.mark.parametrize("nside", [1, 2, 3, 4])
def test_roundtrip_and_equal_area(oracle_lib, nside):
    z, phi = centres(oracle_lib, nside)
    npix = z.size
    for p in range(npix):
        assert ang2pix_ring(nside, z[p], phi[p]) == p
    # equal area: a fine equal-area lattice (uniform in z and phi) binned by
    # the inverse map gives 4 pi / npix per pixel up to lattice error
    nz, nphi = 720, 1440
    zz = -1 + (np.arange(nz) + 0.5) * 2.0 / nz
    pp = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    counts = np.zeros(npix)
    for zv in zz:
        for pv in pp:
            counts[ang2pix_ring(nside, zv, pv)] += 1
    frac = counts / counts.sum() * npix
    assert np.all(np.abs(frac - 1.0) < 0.03)


def test_los_triad(oracle_lib):
    """n, e_l, e_b are orthonormal and right-handed (n x e_l = e_b); l = phi,
    b = pi/2 - theta; the Galactic centre direction (l = 0, b = 0) is +x."""
    for nside in (1, 4):
        for p in range(12 * nside * nside):
            t = oracle_lib.los(nside, p)
            n, el, eb = t["n"], t["el"], t["eb"]
            M = np.stack([n, el, eb])
            assert np.allclose(M @ M.T, np.eye(3), atol=1e-14)
            assert np.allclose(np.cross(n, el), eb, atol=1e-14)
            z, phi = oracle_lib.healpix_centre(nside, p)
            assert t["l"] == pytest.approx(phi, abs=1e-15)
            assert math.sin(t["b"]) == pytest.approx(z, abs=1e-14)
    t = oracle_lib.los(1, 4)   # equatorial pixel at phi = 0
    assert np.allclose(t["n"], [1, 0, 0], atol=1e-15)


@pytest.mark.parametrize("nside", [1024, 8192])
def test_roundtrip_large_nside(oracle_lib, nside):
    """Up to Nside 8192 (the largest the library takes): sampled centres map
    back to their own index under the independent inverse map, at both
    poles, across both cap/belt boundaries, on the equator and at random."""
    npix = 12 * nside * nside
    ncap = 2 * nside * (nside - 1)
    runs = [range(0, 200), range(ncap - 100, ncap + 100), range(npix // 2 - 100, npix // 2 + 100),
            range(npix - ncap - 100, npix - ncap + 100), range(npix - 200, npix)]
    rng = np.random.default_rng(nside)
    pix = list(rng.integers(0, npix, 2000)) + [p for r in runs for p in r]
    for p in pix:
        z, phi = oracle_lib.healpix_centre(nside, int(p))
        assert -1.0 < z < 1.0 and 0.0 <= phi < 2 * math.pi
        assert ang2pix_ring(nside, z, phi) == p
