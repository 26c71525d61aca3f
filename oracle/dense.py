"""Explicit sparse/dense Wilson-clover matrix, assembled site by site (tiny lattices).

Test infrastructure only (see the package docstring).

Block (x, y) of A, with 12x12 blocks indexed by (spin, colour) -> 3*spin + colour:
  diagonal:        1/(2 kappa) * 1 + D_cl(x)
  y = x + mu_hat:  -1/2 (1 - gamma_mu) (x) U_mu(x)          (times -1 if the hop wraps in t)
  y = x - mu_hat:  -1/2 (1 + gamma_mu) (x) U_mu(x - mu)^dag  (times -1 if the hop wraps in t)
This is Eq. 1-3 written as a matrix; it does not call the vectorised operator.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import wilson as W


def site_index(x, y, z, t, dims):
    Lx, Ly, Lz, Lt = dims
    return (x % Lx) + Lx * ((y % Ly) + Ly * ((z % Lz) + Lz * (t % Lt)))


def assemble_A(U: np.ndarray, kappa: float, csw: float, bc_t: float = -1.0) -> sp.csr_matrix:
    Lt, Lz, Ly, Lx = U.shape[:4]
    dims = (Lx, Ly, Lz, Lt)
    V = Lx * Ly * Lz * Lt
    g = W.gammas()
    one = np.eye(4, dtype=np.complex128)
    rows, cols, vals = [], [], []

    def put(i, j, B):
        r, c = np.nonzero(np.abs(B) > 0)
        rows.extend(12 * i + r)
        cols.extend(12 * j + c)
        vals.extend(B[r, c])

    link = lambda c, mu: U[(c[3] % Lt, c[2] % Lz, c[1] % Ly, c[0] % Lx, mu)]
    for t in range(Lt):
        for z in range(Lz):
            for y in range(Ly):
                for x in range(Lx):
                    c = (x, y, z, t)
                    i = site_index(x, y, z, t, dims)
                    diag = np.eye(12, dtype=np.complex128) / (2 * kappa)
                    if csw != 0.0:
                        acc = np.zeros((12, 12), dtype=np.complex128)
                        for mu in range(4):
                            for nu in range(4):
                                if mu != nu:
                                    Fmn = W._leaves_at(link, c, mu, nu) - W._leaves_at(link, c, nu, mu)
                                    acc += np.kron(g[mu] @ g[nu], Fmn)
                        diag = diag - (csw / 32.0) * acc
                    put(i, i, diag)
                    for mu in range(4):
                        cf = list(c)
                        cf[mu] += 1
                        sf = bc_t if (mu == 3 and cf[3] == Lt) else 1.0
                        put(i, site_index(*cf, dims), -0.5 * sf * np.kron(one - g[mu], link(c, mu)))
                        cb = list(c)
                        cb[mu] -= 1
                        sb = bc_t if (mu == 3 and cb[3] == -1) else 1.0
                        put(i, site_index(*cb, dims),
                            -0.5 * sb * np.kron(one + g[mu], link(cb, mu).conj().T))
    return sp.coo_matrix((vals, (rows, cols)), shape=(12 * V, 12 * V)).tocsr()


def to_flat(psi: np.ndarray) -> np.ndarray:
    """Canonical spinor (Lt, Lz, Ly, Lx, 4, 3) -> vector ordered (site, spin, colour)."""
    return psi.reshape(-1)


def from_flat(v: np.ndarray, dims) -> np.ndarray:
    Lx, Ly, Lz, Lt = dims
    return v.reshape(Lt, Lz, Ly, Lx, 4, 3)
