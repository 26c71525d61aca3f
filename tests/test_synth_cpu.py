"""The seeded input generator (shared by the oracle and the GPU side): its 3x3 products,
matrix exponential, SU(3) projection and APE smearing, pinned against library routines
and the group's defining properties."""
import numpy as np
import pytest
import torch

import synth
from synth.gauge import _expi_hermitian, gell_mann, mm3, reunitarize


def _rand_c(n, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.complex(torch.randn(n, 3, 3, generator=g, dtype=torch.float64),
                         torch.randn(n, 3, 3, generator=g, dtype=torch.float64))


def test_mm3_is_the_matrix_product():
    A, B = _rand_c(64, 1), _rand_c(64, 2)
    assert torch.allclose(mm3(A, B), A @ B, rtol=0, atol=1e-13)


def test_exponential_matches_expm():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(3)
    eta = rng.standard_normal((16, 8)) * 1.7      # large enough to need several squarings
    H = np.einsum("na,aij->nij", eta, gell_mann()) * 0.5
    got = _expi_hermitian(torch.from_numpy(H)).numpy()
    for n in range(16):
        want = scipy_linalg.expm(1j * H[n])
        assert np.abs(got[n] - want).max() <= 1e-13


def test_random_field_is_su3_and_seeded():
    dims = (4, 4, 2, 2)
    U = synth.random_su3_field(dims, 0.6, 9)
    W = U.reshape(-1, 3, 3)
    eye = torch.eye(3, dtype=W.dtype)
    assert float((mm3(W, W.conj().transpose(-1, -2)) - eye).abs().max()) <= 1e-14
    assert float((torch.linalg.det(W) - 1).abs().max()) <= 1e-14
    assert torch.equal(U, synth.random_su3_field(dims, 0.6, 9))
    assert not torch.equal(U, synth.random_su3_field(dims, 0.6, 10))


def test_reunitarize_is_identity_on_su3_and_projects_otherwise():
    U = synth.random_su3_field((2, 2, 2, 2), 0.4, 4).reshape(-1, 3, 3)
    assert float((reunitarize(U) - U).abs().max()) <= 1e-14
    M = U + 0.1 * _rand_c(U.shape[0], 5)
    P = reunitarize(M)
    eye = torch.eye(3, dtype=P.dtype)
    assert float((mm3(P, P.conj().transpose(-1, -2)) - eye).abs().max()) <= 1e-14
    assert float((torch.linalg.det(P) - 1).abs().max()) <= 1e-14


def _plaquette(U):
    """Mean of Re tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag / 3 over all planes."""
    from synth.gauge import _sh
    tot, n = 0.0, 0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Um, Un = U[..., mu, :, :], U[..., nu, :, :]
            P = mm3(mm3(Um, _sh(Un, mu, 1)), mm3(_sh(Um, nu, 1), Un).conj().transpose(-1, -2))
            tot += float(P.diagonal(dim1=-2, dim2=-1).sum(-1).real.mean()) / 3
            n += 1
    return tot / n


def test_ape_smearing_keeps_su3_and_smooths():
    U = synth.random_su3_field((4, 4, 4, 4), 0.6, 12)
    S = synth.ape_smear(U, 0.5, 2)
    W = S.reshape(-1, 3, 3)
    eye = torch.eye(3, dtype=W.dtype)
    assert float((mm3(W, W.conj().transpose(-1, -2)) - eye).abs().max()) <= 1e-13
    assert float((torch.linalg.det(W) - 1).abs().max()) <= 1e-13
    assert _plaquette(S) > _plaquette(U) + 0.05
    # the unit field is a fixed point
    one = synth.unit_gauge((4, 4, 2, 2))
    assert float((synth.ape_smear(one, 0.5, 1) - one).abs().max()) <= 1e-14
