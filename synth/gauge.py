"""Random SU(3) gauge fields and APE smearing (input generation only).

Canonical layout everywhere in this project: a gauge field is a complex128 array of
shape (Lt, Lz, Ly, Lx, 4, 3, 3); index [t, z, y, x, mu, a, b] is the colour matrix
element (a, b) of the forward link U_mu(x) that joins site x to x + mu_hat, with
mu = 0, 1, 2, 3 for x, y, z, t.  The field is periodic in every direction; the
fermion boundary condition in time is not part of the gauge field.

Heavy steps (matrix exponential, smearing) run in torch FP64 on any device so that
the 2M-site workloads can be built on a GPU in seconds; the random numbers are always
drawn on the host with PCG64, so the field is the same on every device up to the
rounding of those steps.
"""
from __future__ import annotations

import math

import numpy as np
import torch

# Gell-Mann matrices lambda_1 .. lambda_8 (standard normalisation tr(l_a l_b) = 2 delta_ab).
_GM = np.zeros((8, 3, 3), dtype=np.complex128)
_GM[0][0, 1] = _GM[0][1, 0] = 1
_GM[1][0, 1] = -1j
_GM[1][1, 0] = 1j
_GM[2][0, 0] = 1
_GM[2][1, 1] = -1
_GM[3][0, 2] = _GM[3][2, 0] = 1
_GM[4][0, 2] = -1j
_GM[4][2, 0] = 1j
_GM[5][1, 2] = _GM[5][2, 1] = 1
_GM[6][1, 2] = -1j
_GM[6][2, 1] = 1j
_GM[7][0, 0] = _GM[7][1, 1] = 1 / np.sqrt(3)
_GM[7][2, 2] = -2 / np.sqrt(3)


def gell_mann() -> np.ndarray:
    return _GM.copy()


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def reunitarize(M: torch.Tensor) -> torch.Tensor:
    """Project [..., 3, 3] complex matrices onto SU(3) by Gram-Schmidt on the rows.

    Row 0 is normalised, row 1 is orthogonalised against it and normalised, and row 2
    is set to conj(row0 x row1), which makes the determinant exactly one.
    """
    r0 = M[..., 0, :]
    r0 = r0 / torch.linalg.vector_norm(r0, dim=-1, keepdim=True)
    r1 = M[..., 1, :]
    r1 = r1 - (r0.conj() * r1).sum(-1, keepdim=True) * r0
    r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
    r2 = torch.stack([
        r0[..., 1] * r1[..., 2] - r0[..., 2] * r1[..., 1],
        r0[..., 2] * r1[..., 0] - r0[..., 0] * r1[..., 2],
        r0[..., 0] * r1[..., 1] - r0[..., 1] * r1[..., 0],
    ], dim=-1).conj()
    return torch.stack([r0, r1, r2], dim=-2)


def mm3(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """Products of [..., 3, 3] matrices as one broadcast multiply and a sum over the inner
    index: elementwise kernels, which run at memory speed for millions of 3x3 matrices
    where a batched GEMM of that shape is two orders of magnitude slower."""
    return (A.unsqueeze(-1) * B.unsqueeze(-3)).sum(-2)


def _dag(M: torch.Tensor) -> torch.Tensor:
    return M.conj().transpose(-1, -2)


def _expi_hermitian(Hm: torch.Tensor, terms: int = 18) -> torch.Tensor:
    """exp(i H) for Hermitian [..., 3, 3] H by scaling and squaring: X = i H / 2^s with
    |X|_F <= 1/2, a Taylor polynomial of X (Horner form, remainder < 1e-20), then s
    squarings.  Batched matrix products only, so it runs on any device."""
    nrm = float(torch.linalg.matrix_norm(Hm).max()) if Hm.numel() else 0.0
    s = max(0, math.ceil(math.log2(nrm / 0.5))) if nrm > 0.5 else 0
    X = (1j / 2 ** s) * Hm
    eye = torch.eye(3, dtype=Hm.dtype, device=Hm.device).expand_as(Hm)
    E = eye.clone()
    for n in range(terms, 0, -1):
        E = eye + mm3(X, E) / n
    for _ in range(s):
        E = mm3(E, E)
    return E


def random_su3_field(dims, width: float, seed: int, device="cpu", chunk=1 << 20) -> torch.Tensor:
    """U = reunitarise(exp(i * width * sum_a eta_a lambda_a / 2)), eta_a ~ N(0, 1).

    dims = (Lx, Ly, Lz, Lt).  Returns complex128 (Lt, Lz, Ly, Lx, 4, 3, 3) on `device`.
    """
    Lx, Ly, Lz, Lt = dims
    n = Lx * Ly * Lz * Lt * 4
    eta = _rng(seed).standard_normal(size=(n, 8))
    gm = torch.from_numpy(_GM).to(device)
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    for s in range(0, n, chunk):
        e = torch.from_numpy(eta[s:s + chunk]).to(device).to(torch.complex128)
        Hm = 0.5 * width * torch.einsum("na,aij->nij", e, gm)
        out[s:s + chunk] = reunitarize(_expi_hermitian(Hm))
    return out.reshape(Lt, Lz, Ly, Lx, 4, 3, 3)


def unit_gauge(dims, device="cpu") -> torch.Tensor:
    Lx, Ly, Lz, Lt = dims
    eye = torch.eye(3, dtype=torch.complex128, device=device)
    return eye.expand(Lt, Lz, Ly, Lx, 4, 3, 3).clone()


_AX = (3, 2, 1, 0)  # direction mu (x, y, z, t) -> array axis of the (t, z, y, x) site block


def _sh(F: torch.Tensor, mu: int, step: int) -> torch.Tensor:
    """F(x + step * mu_hat) for a per-site field, periodic."""
    return torch.roll(F, shifts=-step, dims=_AX[mu])


def ape_smear(U: torch.Tensor, alpha: float = 0.5, steps: int = 5) -> torch.Tensor:
    """APE smearing: U'_mu = Proj[(1 - alpha) U_mu + alpha/6 * sum_{nu != mu} staples].

    All links are updated simultaneously in each step; Proj is the Gram-Schmidt
    reunitarisation above (the workload text leaves the projection open).
    """
    for _ in range(steps):
        new = torch.empty_like(U)
        for mu in range(4):
            Umu = U[..., mu, :, :]
            S = torch.zeros_like(Umu)
            for nu in range(4):
                if nu == mu:
                    continue
                Unu = U[..., nu, :, :]
                # upper staple U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
                S = S + mm3(mm3(Unu, _sh(Umu, nu, 1)), _dag(_sh(Unu, mu, 1)))
                # lower staple U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
                Unm = _sh(Unu, nu, -1)
                S = S + mm3(mm3(_dag(Unm), _sh(Umu, nu, -1)), _sh(Unm, mu, 1))
            new[..., mu, :, :] = reunitarize((1 - alpha) * Umu + (alpha / 6.0) * S)
        U = new
    return U
