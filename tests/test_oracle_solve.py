"""Whole-solve pin: the oracle's SAP-FGMRES-DR against a brute-force sparse LU on 4^4."""
import numpy as np
import scipy.sparse.linalg as spl

import synth
from oracle import dense as DN
from oracle import solve as S


def test_solve_matches_direct_lu_4x4():
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.6, 41).numpy()
    f = synth.gaussian_source(dims, 42)
    kappa, csw = 0.13, 1.0
    x, info = S.solve(U, f, kappa, csw, (2, 2, 2, 2), 4, 4, m=8, k=2, tol=1e-10)
    A = DN.assemble_A(U, kappa, csw).tocsc()
    xl = spl.spsolve(A, f.ravel())
    assert S.true_residual(U, x, f, kappa, csw) <= 1e-10
    # |x - x_LU| / |x_LU| <= cond(A) * 1e-10; cond(A) of this operator is O(10)
    assert np.linalg.norm(x.ravel() - xl) <= 1e-8 * np.linalg.norm(xl)
