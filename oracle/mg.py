"""Oracle for the Schwarz method as the smoother of a two-level aggregation multigrid
preconditioner.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper mentions this use of its domain-decomposition preconditioner only among related
work (Sec. V: algebraic multigrid methods that use a Schwarz method as their smoother,
Frommer et al. and Luescher).  It does not define the multigrid method, so the steps here
restate the two-level aggregation method of those works in its plainest form:

  * aggregates: the lattice cut into blocks of a_x x a_y x a_z x a_t sites.  Each aggregate
    and each chirality (spins 0, 1: gamma_5 = +1; spins 2, 3: gamma_5 = -1 in the chiral
    basis of the operator) carries n_tv coarse degrees of freedom, so the interpolation
    commutes with gamma_5;
  * test vectors: n_tv fields v_k, each replaced `setup_iters` times either by M_sap v_k
    (mode "inverse": the Schwarz method as an approximate inverse) or by v_k - M_sap A v_k
    (mode "nullspace": one Schwarz cycle set on A v = 0 from v_k, the smoother's error
    propagator, which removes what the smoother resolves and keeps the low modes of A);
  * interpolation P: on every (aggregate, chirality) the pieces of v_1 .. v_n made
    orthonormal in order (the Q of a QR factorisation whose R has a positive diagonal);
  * coarse operator: D_c = P^H A P (Galerkin);
  * one application of the preconditioner to b: e_c = D_c^{-1} P^H b, x = P e_c, then
    I_Schwarz cycles of the Schwarz method on what is left, x <- x + M_sap (b - A x).

Layouts.  P is held as n_tv fields in the canonical spinor layout (Lt, Lz, Ly, Lx, 4, 3):
field k restricted to an aggregate and to the spins of chirality c is that aggregate's
column (c, k) (the two chiralities have disjoint supports, so one field holds both).
A coarse vector has shape (Nt, Nz, Ny, Nx, 2, n_tv) with N_mu = L_mu / a_mu: aggregate
(x fastest), chirality, test vector.
"""
from __future__ import annotations

import numpy as np

from . import dd as DD
from . import wilson as W

CHIRAL_SPINS = ((0, 1), (2, 3))   # gamma_5 = diag(1, 1, -1, -1)


class Aggregates:
    """Blocks of a = (a_x, a_y, a_z, a_t) sites; a_mu divides L_mu."""

    def __init__(self, dims, a):
        self.dims = tuple(int(v) for v in dims)
        self.a = tuple(int(v) for v in a)
        for L, b in zip(self.dims, self.a):
            if b < 1 or L % b:
                raise ValueError(f"aggregate extent {b} does not divide {L}")
        self.cdims = tuple(L // b for L, b in zip(self.dims, self.a))   # (Nx, Ny, Nz, Nt)
        self.n = int(np.prod(self.cdims))
        Lx, Ly, Lz, Lt = self.dims
        t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
        Nx, Ny, Nz, _ = self.cdims
        ax, ay, az, at = self.a
        # aggregate of every site, lexicographic with x fastest
        self.index = (x // ax) + Nx * ((y // ay) + Ny * ((z // az) + Nz * (t // at)))

    def sum_blocks(self, s: np.ndarray) -> np.ndarray:
        """Sum a per-site array s[t, z, y, x, ...] over every aggregate -> [Nt, Nz, Ny, Nx, ...]."""
        Lx, Ly, Lz, Lt = self.dims
        ax, ay, az, at = self.a
        Nx, Ny, Nz, Nt = self.cdims
        r = s.reshape((Nt, at, Nz, az, Ny, ay, Nx, ax) + s.shape[4:])
        return r.sum(axis=(1, 3, 5, 7))

    def spread(self, c: np.ndarray) -> np.ndarray:
        """Per-aggregate array c[Nt, Nz, Ny, Nx, ...] -> per-site array (each site gets its aggregate's value)."""
        ax, ay, az, at = self.a
        return np.repeat(np.repeat(np.repeat(np.repeat(c, at, axis=0), az, axis=1), ay, axis=2), ax, axis=3)


def interpolation(tv, agg: Aggregates) -> np.ndarray:
    """P from the test vectors: per (aggregate, chirality) the pieces of v_1..v_n made
    orthonormal in order.  Returns an array (n_tv, Lt, Lz, Ly, Lx, 4, 3)."""
    V = np.asarray(tv, dtype=np.complex128)
    ntv = V.shape[0]
    P = np.zeros_like(V)
    flat_idx = agg.index.ravel()
    Vs = V.reshape(ntv, -1, 4, 3)              # (k, site, spin, colour)
    Ps = P.reshape(ntv, -1, 4, 3)
    for X in range(agg.n):
        sites = np.nonzero(flat_idx == X)[0]
        for spins in CHIRAL_SPINS:
            blk = Vs[:, sites][:, :, list(spins), :].reshape(ntv, -1).T      # (6 |X|, n_tv)
            if blk.shape[0] < ntv:
                raise ValueError("more test vectors than degrees of freedom per aggregate and chirality")
            Q, R = np.linalg.qr(blk)
            ph = np.diag(R) / np.abs(np.diag(R))                              # make diag(R) > 0
            Q = Q * ph[None, :]
            q = Q.T.reshape(ntv, len(sites), 2, 3)
            for i, s in enumerate(spins):
                Ps[:, sites, s, :] = q[:, :, i, :]
    return P


def restrict(P: np.ndarray, agg: Aggregates, r: np.ndarray) -> np.ndarray:
    """P^H r: coarse vector (Nt, Nz, Ny, Nx, 2, n_tv)."""
    ntv = P.shape[0]
    out = np.zeros(agg.cdims[::-1] + (2, ntv), dtype=np.complex128)
    for c, spins in enumerate(CHIRAL_SPINS):
        for k in range(ntv):
            site = np.einsum("tzyxsc,tzyxsc->tzyx", P[k][..., list(spins), :].conj(), r[..., list(spins), :])
            out[..., c, k] = agg.sum_blocks(site)
    return out


def prolong(P: np.ndarray, agg: Aggregates, e: np.ndarray) -> np.ndarray:
    """P e: fine field from a coarse vector."""
    ntv = P.shape[0]
    x = np.zeros(P.shape[1:], dtype=np.complex128)
    for c, spins in enumerate(CHIRAL_SPINS):
        for k in range(ntv):
            w = agg.spread(e[..., c, k])
            for s in spins:
                x[..., s, :] += w[..., None] * P[k][..., s, :]
    return x


def coarse_matrix(U, kappa, csw, P: np.ndarray, agg: Aggregates, F=None) -> np.ndarray:
    """D_c = P^H A P as a dense matrix over the flattened coarse vectors: column (Y, c, k) is
    P^H A applied to the interpolation column of aggregate Y, chirality c, test vector k."""
    if F is None and csw != 0.0:
        F = W.field_strength(U)
    ntv = P.shape[0]
    nc = agg.n * 2 * ntv
    D = np.zeros((nc, nc), dtype=np.complex128)
    for Y in range(agg.n):
        mask = (agg.index == Y)
        for c, spins in enumerate(CHIRAL_SPINS):
            for k in range(ntv):
                col = np.zeros_like(P[k])
                for s in spins:
                    col[..., s, :] = np.where(mask[..., None], P[k][..., s, :], 0.0)
                D[:, (Y * 2 + c) * ntv + k] = restrict(P, agg, W.apply_A(U, col, kappa, csw, F)).ravel()
    return D


def two_level(U, kappa, csw, P, agg: Aggregates, Dc, b, dom: DD.Domains, i_schwarz: int, i_domain: int,
              F=None, solver=None):
    """One application of the two-level preconditioner to b (exact coarse solve)."""
    if F is None and csw != 0.0:
        F = W.field_strength(U)
    ec = np.linalg.solve(Dc, restrict(P, agg, b).ravel()).reshape(agg.cdims[::-1] + (2, P.shape[0]))
    x = prolong(P, agg, ec)
    if i_schwarz > 0:
        r = b - W.apply_A(U, x, kappa, csw, F)
        x = x + DD.sap(U, F, r, kappa, csw, dom, i_schwarz, i_domain, solver=solver)
    return x


def smooth_test_vectors(U, kappa, csw, tv0, setup_iters: int, dom: DD.Domains, i_schwarz: int, i_domain: int,
                        mode: str = "inverse", F=None, solver=None):
    """The test vectors after `setup_iters` smoothing steps (see the module docstring)."""
    if mode not in ("inverse", "nullspace"):
        raise ValueError(mode)
    if F is None and csw != 0.0:
        F = W.field_strength(U)
    if solver is None and setup_iters > 0:
        solver = DD.BlockSolver(U, F, kappa, csw, dom)
    tv = [np.array(v, dtype=np.complex128) for v in tv0]
    for _ in range(setup_iters):
        if mode == "inverse":
            tv = [DD.sap(U, F, v, kappa, csw, dom, i_schwarz, i_domain, solver=solver) for v in tv]
        else:
            tv = [v - DD.sap(U, F, W.apply_A(U, v, kappa, csw, F), kappa, csw, dom, i_schwarz, i_domain,
                             solver=solver) for v in tv]
    return tv


def setup(U, kappa, csw, tv0, agg: Aggregates, setup_iters: int, dom: DD.Domains, i_schwarz: int, i_domain: int,
          F=None, solver=None, mode: str = "inverse"):
    """Test vectors smoothed by the Schwarz method, the interpolation and D_c.
    Returns (P, Dc)."""
    if F is None and csw != 0.0:
        F = W.field_strength(U)
    tv = smooth_test_vectors(U, kappa, csw, tv0, setup_iters, dom, i_schwarz, i_domain, mode, F, solver)
    P = interpolation(tv, agg)
    return P, coarse_matrix(U, kappa, csw, P, agg, F)
