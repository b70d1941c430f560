"""The low-order surrogate basis (real spherical harmonics at the pixel
centres, orthonormalised by CholeskyQR2; SYNAX_SUR_BASIS_SH) on the GPU
against the oracle's basis (oracle/surrogate.py: scipy's associated Legendre
functions, numpy's Cholesky), and the surrogate's projection with it.

Tolerances: the basis in FP64, 1e-9 absolute per entry (both sides are
exact constructions in double; the Gram matrices differ by rounding only);
projections through the BF16 hi + lo split, 3e-5 of the map norm.
"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import surrogate as osur
from paper_2410_01136_gb300 import _native, forward, inputs
from paper_2410_01136_gb300.surrogate import Surrogate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_01136_gb300 import build
    build()
    oracle.build()
    return _t


def gpu_basis(torch, nside, nb):
    out = torch.empty((nb, 12 * nside * nside), dtype=torch.float64, device="cuda")
    _native.check(_native.lib().synax_sh_basis(nside, nb, ctypes.c_void_p(out.data_ptr())), "synax_sh_basis")
    return out


@pytest.mark.parametrize("nside,nb", [(4, 64), (16, 1024)])
def test_basis_matches_oracle(torch, nside, nb):
    E = gpu_basis(torch, nside, nb).cpu().numpy()
    ref = osur.sh_basis(nside, nb)
    np.testing.assert_allclose(E, ref, rtol=0, atol=1e-9)


def test_basis_orthonormal_at_nside64(torch):
    E = gpu_basis(torch, 64, 3072)
    G = E @ E.T
    err = (G - torch.eye(3072, dtype=torch.float64, device="cuda")).abs().max().item()
    assert err < 1e-10, err
    # the monopole row is the constant map
    np.testing.assert_allclose(E[0].cpu().numpy(), 1.0 / np.sqrt(49152), rtol=1e-12)


def small_sh_surrogate(nside=16, nb=1024, **kw):
    lo, hi = inputs.config5_box()
    sur = Surrogate(16, lo, hi, None, None, basis="sh", n_basis=nb, nside=nside, width=256, depth=2, batch=128,
                    max_eval=512, map_chunk=16, **kw)
    sur.set_params(inputs.mlp_init(sur.widths, seed=7))
    return sur


def test_projection_matches_oracle(torch):
    nside, nb = 16, 1024
    sur = small_sh_surrogate(nside, nb)
    prob = inputs.config5_problem().replace(nside=nside, n_steps=128)
    maps = forward(prob)                                 # [1, 3, npix]
    c = sur.project(maps.reshape(3, -1)).cpu().numpy()
    E = osur.sh_basis(nside, nb)
    x = maps.reshape(3, -1).double().cpu().numpy()
    ref = x @ E.T
    for s in range(3):
        assert np.abs(c[s] - ref[s]).max() <= 3e-5 * np.linalg.norm(x[s]), s
    # Parseval inside the basis: the truncation is what the basis leaves out
    trunc = np.sum(x * x, axis=1) - np.sum(ref * ref, axis=1)
    assert np.all(trunc >= -1e-9 * np.sum(x * x, axis=1))
    sur.close()


def test_sh_surrogate_trains(torch):
    nside, nb = 16, 1024
    sur = small_sh_surrogate(nside, nb, total_steps=60, lr=1e-3)
    prob = inputs.config5_problem().replace(nside=nside, n_steps=64)
    th = inputs.config5_thetas(256, seed=52)
    sur.dataset(prob, th)
    losses = sur.train(60, seed=3)
    assert np.all(np.isfinite(losses)) and losses[-10:].mean() < losses[:10].mean()
    c, rms, fell = sur.judge(prob, th[:8], sur(torch.tensor(th[:8], dtype=torch.float32, device="cuda")), 1.0)
    assert np.all(np.isfinite(rms.cpu().numpy()))
    sur.close()
