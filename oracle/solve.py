"""Oracle for the whole solve of Table I: FGMRES-DR outer solver, multiplicative SAP
preconditioner with MR domain solves, everything in FP64.  Test infrastructure only."""
from __future__ import annotations

import numpy as np

from . import dd as DD
from . import fgmres as FG
from . import wilson as W


def solve(U, f, kappa, csw, domain, i_schwarz, i_domain, m, k, tol=1e-10, max_cycles=100):
    """Return (x, info): A x = f to |f - A x| / |f| <= tol."""
    dims = (U.shape[3], U.shape[2], U.shape[1], U.shape[0])
    F = W.field_strength(U) if csw != 0.0 else None
    dom = DD.Domains(dims, domain)
    bs = DD.BlockSolver(U, F, kappa, csw, dom)
    shape = f.shape
    A = lambda v: W.apply_A(U, v.reshape(shape), kappa, csw, F).ravel()
    M = lambda v: DD.sap(U, F, v.reshape(shape), kappa, csw, dom, i_schwarz, i_domain, solver=bs).ravel()
    x, info = FG.fgmres_dr(A, M, f.ravel(), m, k, tol=tol, max_cycles=max_cycles)
    return x.reshape(shape), info


def true_residual(U, x, f, kappa, csw) -> float:
    """|f - A x| / |f| in FP64."""
    r = f - W.apply_A(U, x, kappa, csw)
    return float(np.linalg.norm(r) / np.linalg.norm(f))
