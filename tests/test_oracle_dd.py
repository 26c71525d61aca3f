"""Pins for the oracle's domain decomposition, Schur complement, MR and SAP (Sec. II-D)."""
import numpy as np
import pytest

import synth
from oracle import dd as DD
from oracle import dense as DN
from oracle import wilson as W

DIMS = (4, 4, 4, 4)
B2 = (2, 2, 2, 2)


@pytest.fixture(scope="module")
def small():
    U = synth.random_su3_field(DIMS, 0.6, 31).numpy()
    F = W.field_strength(U)
    f = synth.gaussian_source(DIMS, 32)
    return U, F, f


def test_domain_shape_validation():
    with pytest.raises(ValueError):
        DD.Domains((8, 8, 8, 8), (8, 4, 4, 4))   # L/b = 1 in x
    with pytest.raises(ValueError):
        DD.Domains((12, 8, 8, 8), (4, 4, 4, 4))  # L/b = 3 (odd) in x
    with pytest.raises(ValueError):
        DD.Domains((6, 8, 8, 8), (3, 4, 4, 4))   # odd extent


def test_colouring_is_checkerboard():
    dom = DD.Domains((8, 8, 8, 8), (4, 4, 4, 4))
    for mu in range(4):
        for s in (1, -1):
            cross = ~dom.same_domain(mu, s)
            nb = W.shift(dom.colour, mu, s)
            assert np.all(dom.colour[cross] != nb[cross])


def test_D_plus_R_is_A(small):
    U, F, f = small
    dom = DD.Domains(DIMS, B2)
    a = W.apply_A(U, f, 0.13, 1.2, F)
    assert np.abs(DD.apply_D(U, F, f, 0.13, 1.2, dom) + DD.apply_R(U, f, dom) - a).max() < 1e-13


def test_D_is_block_diagonal_and_R_off_block(small):
    U, F, f = small
    dom = DD.Domains(DIMS, B2)
    for d in (0, 5, 11):
        m = (dom.domain == d)[..., None, None]
        Df = DD.apply_D(U, F, f * m, 0.13, 1.2, dom)
        assert np.abs(Df * ~m).max() == 0
        Rf = DD.apply_R(U, f * m, dom)
        assert np.abs(Rf * m).max() == 0


def test_schur_identity(small):
    U, F, f = small
    dom = DD.Domains(DIMS, B2)
    bs = DD.BlockSolver(U, F, 0.13, 1.2, dom)
    xe = f * bs.even
    xo = -DD.apply_site_matrix(bs.Dinv, bs.odd * bs.hop_in(xe)) * bs.odd
    full = DD.apply_D(U, F, xe + xo, 0.13, 1.2, dom)
    assert np.abs(full * bs.odd).max() < 1e-13
    assert np.abs(full * bs.even - bs.schur(xe)).max() < 1e-13


def test_even_odd_route_reaches_exact_block_solve(small):
    U, F, f = small
    dom = DD.Domains(DIMS, B2)
    bs = DD.BlockSolver(U, F, 0.13, 1.2, dom)
    ex = DD.ExactBlockSolver(U, F, 0.13, 1.2, dom)
    for colour in (0, 1):
        a = bs.solve(f, colour, 60)
        b = ex.solve(f, colour)
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_mr_one_step_and_monotone(small):
    U, F, f = small
    dom = DD.Domains(DIMS, B2)
    bs = DD.BlockSolver(U, F, 0.13, 1.2, dom)
    cm = (dom.colour == 0)[..., None, None].astype(float)
    fe = f * bs.even * cm
    x1, r1 = bs.mr(fe, cm, 1)
    # closed form after one step, per domain: alpha = <A f, f>/<A f, A f>
    p = bs.schur(fe) * cm
    for d in np.unique(dom.domain[dom.colour == 0]):
        m = (dom.domain == d)[..., None, None]
        a = np.vdot((p * m).ravel(), (fe * m).ravel()) / np.vdot((p * m).ravel(), (p * m).ravel())
        assert np.abs(x1 * m - a * fe * m).max() < 1e-13
    # residual per domain never increases
    prev = None
    for n in range(1, 7):
        _, r = bs.mr(fe, cm, n)
        norms = np.bincount(dom.domain.ravel(), weights=np.sum(np.abs(r) ** 2, axis=(-1, -2)).ravel())
        if prev is not None:
            assert np.all(norms <= prev * (1 + 1e-13))
        prev = norms


def test_mr_exact_on_a_scalar_operator():
    """With every link zero and c_sw = 0 the Schur complement of Eq. 5 is the scalar
    1/(2 kappa) on even sites, so BlockSolver.mr must return x = 2 kappa f after one step
    with a zero residual, and a second step (<p, p> = 0) must leave x unchanged."""
    kappa = 0.13
    U = np.zeros(DIMS[::-1] + (4, 3, 3), dtype=np.complex128)
    dom = DD.Domains(DIMS, B2)
    bs = DD.BlockSolver(U, None, kappa, 0.0, dom)
    f = synth.gaussian_source(DIMS, 33)
    for colour in (0, 1):
        cm = (dom.colour == colour)[..., None, None].astype(float)
        fe = f * bs.even * cm
        for n in (1, 2):
            x, rho = bs.mr(fe, cm, n)
            assert np.abs(x - 2.0 * kappa * fe).max() <= 1e-15 * np.abs(fe).max()
            assert np.abs(rho).max() <= 1e-15 * np.abs(fe).max()


def test_sap_equals_dense_block_gauss_seidel(small):
    U, F, f = small
    dom = DD.Domains(DIMS, B2)
    A = DN.assemble_A(U, 0.13, 1.2).toarray()
    sitedom = np.repeat(dom.domain.ravel(), 12)
    sitecol = np.repeat(dom.colour.ravel(), 12)
    fv = f.ravel()
    u = np.zeros_like(fv)
    for _ in range(3):
        for colour in (0, 1):
            r = fv - A @ u
            for d in np.unique(sitedom[sitecol == colour]):
                idx = np.nonzero(sitedom == d)[0]
                u[idx] += np.linalg.solve(A[np.ix_(idx, idx)], r[idx])
    ex = DD.ExactBlockSolver(U, F, 0.13, 1.2, dom)
    got = DD.sap(U, F, f, 0.13, 1.2, dom, 3, None, solver=ex)
    assert np.linalg.norm(got.ravel() - u) <= 1e-12 * np.linalg.norm(u)


def test_additive_sap_equals_dense_block_jacobi(small):
    """The additive form with exact domain solves is block Jacobi on the dense A: every
    domain solves with the residual of the same iterate (Sec. II-D, Eq. 4)."""
    U, F, f = small
    dom = DD.Domains(DIMS, B2)
    A = DN.assemble_A(U, 0.13, 1.2).toarray()
    sitedom = np.repeat(dom.domain.ravel(), 12)
    fv = f.ravel()
    u = np.zeros_like(fv)
    for _ in range(3):
        r = fv - A @ u
        du = np.zeros_like(u)
        for d in np.unique(sitedom):
            idx = np.nonzero(sitedom == d)[0]
            du[idx] = np.linalg.solve(A[np.ix_(idx, idx)], r[idx])
        u = u + du
    ex = DD.ExactBlockSolver(U, F, 0.13, 1.2, dom)
    got = DD.sap_additive(U, F, f, 0.13, 1.2, dom, 3, None, solver=ex)
    assert np.linalg.norm(got.ravel() - u) <= 1e-12 * np.linalg.norm(u)
    # one sweep of either form is the same block solve of f
    mult = DD.sap(U, F, f, 0.13, 1.2, dom, 1, None, solver=ex)
    add1 = DD.sap_additive(U, F, f, 0.13, 1.2, dom, 1, None, solver=ex)
    black = dom.colour == 0
    assert np.allclose(mult[black], add1[black], rtol=0, atol=1e-14)


def test_sap_converges_to_solution_small_kappa(small):
    U, F, f = small
    dom = DD.Domains(DIMS, B2)
    ex = DD.ExactBlockSolver(U, F, 0.10, 1.2, dom)
    A = DN.assemble_A(U, 0.10, 1.2)
    import scipy.sparse.linalg as spl
    x = spl.spsolve(A.tocsc(), f.ravel())
    errs = []
    for n in (2, 6, 12):
        u = DD.sap(U, F, f, 0.10, 1.2, dom, n, None, solver=ex)
        errs.append(np.linalg.norm(u.ravel() - x) / np.linalg.norm(x))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-8


def test_sap_reduces_residual_8x4():
    w = synth.WORKLOADS["8^4"]
    U = synth.make_gauge(w).numpy()
    F = W.field_strength(U)
    f = synth.make_sources(w)[0]
    dom = DD.Domains(w.dims, w.domain)
    u = DD.sap(U, F, f, w.kappa, w.csw, dom, 2, w.i_domain)
    r = f - W.apply_A(U, u, w.kappa, w.csw, F)
    assert np.linalg.norm(r) < 0.1 * np.linalg.norm(f)
