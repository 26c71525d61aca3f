"""Pins for the two-level multigrid oracle with the Schwarz smoother (related work, Sec. V).

Each pin checks the oracle against something it does not compute itself: the explicit
sparse matrix of A assembled site by site (oracle.dense), orthonormality and span,
gamma_5-hermiticity, the nearest-neighbour structure of a Galerkin operator, and the
exactness of the coarse correction on the range of P.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import dd as DD
from oracle import dense as DN
from oracle import mg as MG
from oracle import wilson as W

KAPPA, CSW = 0.124, 1.3


@pytest.fixture(scope="module")
def lat4():
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.6, 41).numpy()
    F = W.field_strength(U)
    tv = [synth.gaussian_source(dims, 50 + k) for k in range(3)]
    return dims, U, F, tv


def _P_matrix(P, agg):
    """The interpolation as an explicit sparse matrix (fine dof x coarse dof), one column
    per (aggregate, chirality, test vector), built from the definition."""
    ntv = P.shape[0]
    rows, cols, vals = [], [], []
    idx = agg.index.ravel()
    for k in range(ntv):
        f = P[k].reshape(-1, 4, 3)
        for site in range(f.shape[0]):
            X = idx[site]
            for s in range(4):
                c = 0 if s < 2 else 1
                for col in range(3):
                    v = f[site, s, col]
                    if v != 0:
                        rows.append(12 * site + 3 * s + col)
                        cols.append((X * 2 + c) * ntv + k)
                        vals.append(v)
    n_f = P[0].size
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_f, agg.n * 2 * ntv))


def test_aggregate_extent_validation():
    with pytest.raises(ValueError):
        MG.Aggregates((8, 8, 8, 8), (3, 4, 4, 4))


def test_interpolation_orthonormal_and_spans_test_vectors(lat4):
    dims, U, F, tv = lat4
    agg = MG.Aggregates(dims, (2, 2, 2, 2))
    P = MG.interpolation(tv, agg)
    Pm = _P_matrix(P, agg).toarray()
    G = Pm.conj().T @ Pm
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-13
    # each test vector lies in the range of P: P P^H v = v
    for v in tv:
        x = v.ravel()
        assert np.abs(Pm @ (Pm.conj().T @ x) - x).max() < 1e-12
    # restrict / prolong are P^H and P
    r = synth.gaussian_source(dims, 77)
    assert np.abs(MG.restrict(P, agg, r).ravel() - Pm.conj().T @ r.ravel()).max() < 1e-12
    e = np.random.default_rng(3).standard_normal(agg.n * 2 * len(tv)) + 0j
    assert np.abs(MG.prolong(P, agg, e.reshape(agg.cdims[::-1] + (2, len(tv)))).ravel() - Pm @ e).max() < 1e-12


def test_interpolation_gram_schmidt_order(lat4):
    """Column 1 of an aggregate is the first test vector's piece, normalised (the order of
    Gram-Schmidt), and the first column of every aggregate-chirality is a positive multiple."""
    dims, U, F, tv = lat4
    agg = MG.Aggregates(dims, (2, 2, 2, 2))
    P = MG.interpolation(tv, agg)
    for X in (0, 7):
        m = (agg.index == X)
        for spins in MG.CHIRAL_SPINS:
            v = tv[0][m][:, list(spins), :].ravel()
            p = P[0][m][:, list(spins), :].ravel()
            assert np.abs(p - v / np.linalg.norm(v)).max() < 1e-13


def test_coarse_matrix_is_galerkin_product(lat4):
    dims, U, F, tv = lat4
    agg = MG.Aggregates(dims, (2, 2, 2, 2))
    P = MG.interpolation(tv, agg)
    Dc = MG.coarse_matrix(U, KAPPA, CSW, P, agg, F)
    A = DN.assemble_A(U, KAPPA, CSW)
    Pm = _P_matrix(P, agg)
    ref = (Pm.conj().T @ (A @ Pm)).toarray()
    assert np.abs(Dc - ref).max() < 1e-12 * np.abs(ref).max()


def test_coarse_matrix_gamma5_hermitian(lat4):
    dims, U, F, tv = lat4
    agg = MG.Aggregates(dims, (2, 2, 2, 2))
    P = MG.interpolation(tv, agg)
    Dc = MG.coarse_matrix(U, KAPPA, CSW, P, agg, F)
    ntv = len(tv)
    g5 = np.tile(np.repeat([1.0, -1.0], ntv), agg.n)
    lhs = g5[:, None] * Dc * g5[None, :]
    assert np.abs(lhs - Dc.conj().T).max() < 1e-13 * np.abs(Dc).max()


def test_coarse_matrix_nearest_neighbour():
    """On 8x4x4x4 sites in 2x2x2x2 aggregates the coarse lattice is 4x2x2x2: aggregates two
    apart in x are not neighbours and their block of D_c vanishes exactly; neighbours'
    blocks do not."""
    dims = (8, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.6, 43).numpy()
    tv = [synth.gaussian_source(dims, 60 + k) for k in range(2)]
    agg = MG.Aggregates(dims, (2, 2, 2, 2))
    P = MG.interpolation(tv, agg)
    Dc = MG.coarse_matrix(U, KAPPA, 0.0, P, agg)
    n = 2 * len(tv)
    blk = lambda X, Y: Dc[X * n:(X + 1) * n, Y * n:(Y + 1) * n]
    assert np.abs(blk(0, 2)).max() == 0.0          # x = 0 and x = 2 (two apart)
    assert np.abs(blk(0, 1)).max() > 1e-3          # x neighbours
    assert np.abs(blk(0, 3)).max() > 1e-3          # x neighbours through the boundary
    assert np.abs(blk(0, 0)).max() > 1e-3


def test_full_basis_two_level_is_exact_inverse(lat4):
    """One-site aggregates with six test vectors: P is unitary, so the two-level method with
    an exact coarse solve is A^{-1} (checked against a sparse LU solve), and the smoother
    then sees a zero residual."""
    dims, U, F, _ = lat4
    tv = [synth.gaussian_source(dims, 80 + k) for k in range(6)]
    agg = MG.Aggregates(dims, (1, 1, 1, 1))
    P = MG.interpolation(tv, agg)
    Dc = MG.coarse_matrix(U, KAPPA, CSW, P, agg, F)
    b = synth.gaussian_source(dims, 90)
    dom = DD.Domains(dims, (2, 2, 2, 2))
    x = MG.two_level(U, KAPPA, CSW, P, agg, Dc, b, dom, 1, 4, F)
    A = DN.assemble_A(U, KAPPA, CSW).tocsc()
    ref = spla.spsolve(A, b.ravel())
    assert np.linalg.norm(x.ravel() - ref) < 1e-10 * np.linalg.norm(ref)


def test_coarse_correction_exact_on_range_and_galerkin_orthogonal(lat4):
    dims, U, F, tv = lat4
    agg = MG.Aggregates(dims, (2, 2, 2, 2))
    P = MG.interpolation(tv, agg)
    Dc = MG.coarse_matrix(U, KAPPA, CSW, P, agg, F)
    dom = DD.Domains(dims, (2, 2, 2, 2))
    rng = np.random.default_rng(5)
    shape = agg.cdims[::-1] + (2, len(tv))
    y = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    xf = MG.prolong(P, agg, y)
    b = W.apply_A(U, xf, KAPPA, CSW, F)
    x = MG.two_level(U, KAPPA, CSW, P, agg, Dc, b, dom, 0, 4, F)   # coarse correction alone
    assert np.abs(x - xf).max() < 1e-11 * np.abs(xf).max()
    b2 = synth.gaussian_source(dims, 91)
    x2 = MG.two_level(U, KAPPA, CSW, P, agg, Dc, b2, dom, 0, 4, F)
    res = MG.restrict(P, agg, b2 - W.apply_A(U, x2, KAPPA, CSW, F))
    assert np.abs(res).max() < 1e-12 * np.abs(MG.restrict(P, agg, b2)).max()


def test_smoothed_test_vectors_are_sap_images(lat4):
    """setup() with one smoothing step builds P from M_sap v (the Schwarz oracle), so the
    smoothed vectors lie in the range of P."""
    dims, U, F, tv = lat4
    agg = MG.Aggregates(dims, (2, 2, 2, 2))
    dom = DD.Domains(dims, (2, 2, 2, 2))
    P, Dc = MG.setup(U, KAPPA, CSW, tv, agg, 1, dom, 2, 3, F)
    Pm = _P_matrix(P, agg).toarray()
    for v in tv:
        s = DD.sap(U, F, v, KAPPA, CSW, dom, 2, 3).ravel()
        assert np.abs(Pm @ (Pm.conj().T @ s) - s).max() < 1e-12 * np.abs(s).max()
    assert Dc.shape == (agg.n * 2 * len(tv),) * 2


def test_nullspace_smoothing_is_schwarz_iteration_on_zero_rhs(lat4):
    """Mode "nullspace": v - M_sap A v equals the multiplicative Schwarz iteration on
    A x = 0 started from x = v, written out as block Gauss-Seidel with exact block solves
    (dense blocks of the site-by-site sparse A)."""
    dims, U, F, tv = lat4
    dom = DD.Domains(dims, (2, 2, 2, 2))
    ex = DD.ExactBlockSolver(U, F, KAPPA, CSW, dom)
    got = MG.smooth_test_vectors(U, KAPPA, CSW, tv[:1], 1, dom, 2, 0, "nullspace", F, solver=ex)[0]
    A = DN.assemble_A(U, KAPPA, CSW).toarray()
    x = tv[0].ravel().copy()
    blocks = {}
    for colour in (0, 1):
        for d in np.unique(dom.domain[dom.colour == colour]):
            blocks.setdefault(colour, []).append(np.nonzero(np.repeat((dom.domain == d).ravel(), 12))[0])
    for _ in range(2):
        for colour in (0, 1):
            r = -A @ x
            for idx in blocks[colour]:
                x[idx] += np.linalg.solve(A[np.ix_(idx, idx)], r[idx])
    assert np.abs(got.ravel() - x).max() < 1e-11 * np.abs(x).max()
