"""Pins for the oracle's Wilson-clover operator (Eq. 1-3) against facts the physics fixes."""
import itertools

import numpy as np
import pytest

import synth
from oracle import dense as D
from oracle import wilson as W


def rnd_gauge(dims, seed, width=0.6):
    return synth.random_su3_field(dims, width, seed).numpy()


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def test_gamma_algebra():
    g = W.gammas()
    for mu, nu in itertools.product(range(4), repeat=2):
        ac = g[mu] @ g[nu] + g[nu] @ g[mu]
        assert np.allclose(ac, 2 * np.eye(4) * (mu == nu), atol=1e-15)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
    assert np.allclose(W.gamma5(), np.diag([1, 1, -1, -1]))


def free_field_eigs(dims, kappa):
    """Closed form: A(p) = m + sum(1 - cos p) + i sum gamma sin p, eigenvalues
    a +- i sqrt(sum sin^2 p), each 6-fold; p_t antiperiodic."""
    m = 1 / (2 * kappa) - 4
    out = []
    ranges = [[2 * np.pi * n / L for n in range(L)] for L in dims[:3]]
    ranges.append([(2 * n + 1) * np.pi / dims[3] for n in range(dims[3])])
    for p in itertools.product(*ranges):
        p = np.array(p)
        a = m + np.sum(1 - np.cos(p))
        b = np.sqrt(np.sum(np.sin(p) ** 2))
        out += [a + 1j * b] * 6 + [a - 1j * b] * 6
    return np.array(out)


def _sort(ev):
    ev = np.round(ev, 9)
    return ev[np.lexsort((ev.imag, ev.real))]


def test_free_field_spectrum_dense():
    dims = (2, 4, 2, 4)
    kappa = 0.11
    U = synth.unit_gauge(dims).numpy()
    shape = (dims[3], dims[2], dims[1], dims[0], 4, 3)
    n = int(np.prod(shape))
    cols = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        cols[:, j] = W.apply_A(U, e.reshape(shape), kappa, 1.7).ravel()  # clover vanishes at U = 1
    ev = np.linalg.eigvals(cols)
    ref = free_field_eigs(dims, kappa)
    assert np.allclose(_sort(ev), _sort(ref), atol=1e-10)


def test_free_field_plane_waves_8x4():
    dims = (8, 8, 8, 8)
    kappa = 0.125
    U = synth.unit_gauge(dims).numpy()
    g = W.gammas()
    rng = np.random.default_rng(5)
    t, z, y, x = np.meshgrid(*[np.arange(L) for L in dims[::-1]], indexing="ij")
    for _ in range(4):
        n = rng.integers(0, 8, size=4)
        p = 2 * np.pi * n / 8.0
        p[3] = (2 * n[3] + 1) * np.pi / 8.0
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = phase[..., None, None] * chi
        Ap = (1 / (2 * kappa) - 4 + np.sum(1 - np.cos(p))) * np.eye(4) \
            + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        want = phase[..., None, None] * (Ap @ chi)
        got = W.apply_A(U, psi, kappa, 1.0)
        assert np.abs(got - want).max() < 1e-12


def test_gamma5_hermiticity():
    dims = (4, 4, 4, 4)
    U = rnd_gauge(dims, 7)
    phi = synth.gaussian_source(dims, 8)
    psi = synth.gaussian_source(dims, 9)
    g5 = W.gamma5()
    F = W.field_strength(U)
    lhs = vdot(phi, W.spin_times(g5, W.apply_A(U, W.spin_times(g5, psi), 0.13, 1.5, F)))
    rhs = vdot(W.apply_A(U, phi, 0.13, 1.5, F), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(rhs) * 10


def test_gauge_covariance():
    dims = (4, 4, 4, 4)
    U = rnd_gauge(dims, 10)
    psi = synth.gaussian_source(dims, 11)
    Om = rnd_gauge(dims, 12, width=2.0)[..., 0, :, :]          # one SU(3) per site
    Up = np.empty_like(U)
    for mu in range(4):
        Up[..., mu, :, :] = Om @ U[..., mu, :, :] @ np.conj(np.swapaxes(W.shift(Om, mu, 1), -1, -2))
    psip = np.einsum("...ab,...sb->...sa", Om, psi)
    lhs = W.apply_A(Up, psip, 0.13, 1.5)
    rhs = np.einsum("...ab,...sb->...sa", Om, W.apply_A(U, psi, 0.13, 1.5))
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)


def test_clover_structure():
    dims = (4, 4, 4, 4)
    U = rnd_gauge(dims, 13)
    M = W.clover_matrix(W.field_strength(U), 1.5)
    # block diagonal in chirality (spins 0,1 vs 2,3), each 6x6 block Hermitian
    assert np.abs(M[..., :6, 6:]).max() < 1e-15 and np.abs(M[..., 6:, :6]).max() < 1e-15
    assert np.abs(M - np.conj(np.swapaxes(M, -1, -2))).max() < 1e-14
    assert np.abs(M).max() > 0.1
    Mu = W.clover_matrix(W.field_strength(synth.unit_gauge(dims).numpy()), 1.5)
    assert np.abs(Mu).max() < 1e-15


def test_clover_constant_abelian_field():
    """U_x(x) = diag(exp(i theta_a y)), all other links 1; every xy leaf is
    diag(exp(-i theta_a)), so F_xy = -8 i diag(sin theta_a) and the other planes vanish.
    With gamma_x gamma_y = i sigma_3 (+) i sigma_3 in this basis the clover term is
    -(c_sw/2) diag(sigma_3 (+) sigma_3) (x) diag(sin theta_a) at every site."""
    dims = (4, 4, 4, 4)
    Ly = dims[1]
    theta = 2 * np.pi * np.array([1, 2, -3]) / Ly
    U = synth.unit_gauge(dims).numpy().copy()
    for y in range(Ly):
        U[:, :, y, :, 0] = np.diag(np.exp(1j * theta * y))
    csw = 1.3
    M = W.clover_matrix(W.field_strength(U), csw)
    s3 = np.array([1, -1, 1, -1])
    want = np.diag(np.kron(s3, np.sin(theta)) * (-csw / 2))
    assert np.abs(M - want).max() < 1e-13


def test_antiperiodic_equals_signed_links():
    """Antiperiodic t hops equal periodic hops with the t-links at t = L_t - 1 negated
    (the clover is unchanged because every plaquette through the boundary holds two)."""
    dims = (4, 4, 4, 4)
    U = rnd_gauge(dims, 14)
    psi = synth.gaussian_source(dims, 15)
    Us = U.copy()
    Us[-1, ..., 3, :, :] *= -1
    a = W.apply_A(U, psi, 0.13, 1.2, bc_t=-1.0)
    b = W.apply_A(Us, psi, 0.13, 1.2, bc_t=+1.0)
    assert np.abs(a - b).max() < 1e-13


def test_per_site_matches_vectorised():
    dims = (4, 4, 4, 8)
    U = rnd_gauge(dims, 16)
    psi = synth.gaussian_source(dims, 17)
    A = W.apply_A(U, psi, 0.13, 1.1)
    coords = [(0, 0, 0, 0), (3, 3, 3, 7), (1, 2, 3, 4), (2, 0, 1, 7), (0, 3, 2, 0)]
    got = W.apply_A_at(U, psi, 0.13, 1.1, coords)
    for i, (x, y, z, t) in enumerate(coords):
        assert np.abs(got[i] - A[t, z, y, x]).max() < 1e-13


def test_site_by_site_matrix_matches_operator():
    dims = (4, 2, 2, 4)
    U = rnd_gauge(dims, 18)
    psi = synth.gaussian_source(dims, 19)
    A = D.assemble_A(U, 0.12, 1.4)
    assert np.abs(A @ psi.ravel() - W.apply_A(U, psi, 0.12, 1.4).ravel()).max() < 1e-13
