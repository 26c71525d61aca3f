"""Oracle for the Schwarz preconditioner (Sec. II-D, Eq. 4-5, Table I).

Test infrastructure only (see the package docstring).

Readings of the paper taken here:
  * Domains are hyper-rectangles of shape b = (bx, by, bz, bt); every b_mu is even (so the
    local and global checkerboards agree) and every L_mu / b_mu is even and >= 2 (so the
    two-colouring of domains is consistent under periodic wrap and no hop wraps back into
    its own domain).
  * Colour of the domain with block coordinates n is (sum_mu n_mu) mod 2; colour 0
    ("black") is swept first.  One Schwarz iteration is a black half-sweep followed by a
    white half-sweep.
  * Site parity (x + y + z + t) mod 2; even = 0.
  * D is A with every hop between two different domains dropped; R = A - D.
  * MR (Saad) on the even-site Schur complement of D restricted to a domain, exactly
    I_domain steps from x = 0, alpha = <p, rho> / <p, p> with <a, b> = sum conj(a) b,
    no relaxation; a domain with <p, p> = 0 takes alpha = 0.
  * The multiplicative method is block Gauss-Seidel:
        u_c <- u_c + D_c^{-1} (f - A u)_c,  c = black, then white, u^0 = 0,
    with D_c^{-1} replaced by the even-odd MR approximation.
  * The additive method (Sec. II-D, Eq. 4) is block Jacobi: every domain solves with the
    residual of the same iterate, u <- u + D^{-1} (f - A u), u^0 = 0.
"""
from __future__ import annotations

import numpy as np

from . import wilson as W


class Domains:
    """Domain ids, colours and parities of a lattice split into blocks of shape b."""

    def __init__(self, dims, b):
        self.dims = tuple(int(v) for v in dims)      # (Lx, Ly, Lz, Lt)
        self.b = tuple(int(v) for v in b)
        for L, bb in zip(self.dims, self.b):
            if bb % 2 or L % bb or (L // bb) % 2 or L // bb < 2:
                raise ValueError(f"invalid domain shape {b} for lattice {dims}")
        self.nblk = tuple(L // bb for L, bb in zip(self.dims, self.b))
        Lx, Ly, Lz, Lt = self.dims
        t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                                 indexing="ij")
        self.coords = (x, y, z, t)
        n = [c // bb for c, bb in zip(self.coords, self.b)]
        nx, ny, nz, _ = self.nblk
        self.domain = n[0] + nx * (n[1] + ny * (n[2] + nz * n[3]))
        self.colour = (n[0] + n[1] + n[2] + n[3]) % 2
        self.parity = (x + y + z + t) % 2
        self.ndomains = int(np.prod(self.nblk))

    def same_domain(self, mu: int, step: int) -> np.ndarray:
        """Mask of sites x whose neighbour x + step*mu lies in the same domain."""
        return self.domain == W.shift(self.domain, mu, step)

    def keep_inside(self, mu, step):
        return self.same_domain(mu, step).astype(np.float64)

    def keep_crossing(self, mu, step):
        return (~self.same_domain(mu, step)).astype(np.float64)


def diag_part(F, psi, kappa, csw):
    """Site-diagonal part of A: (1/(2 kappa) + D_cl) psi."""
    out = psi / (2.0 * kappa)
    if csw != 0.0:
        out = out + W.clover_apply(F, psi, csw)
    return out


def apply_D(U, F, psi, kappa, csw, dom: Domains):
    """Block-diagonal part D of A = D + R: hops crossing a domain face dropped."""
    return diag_part(F, psi, kappa, csw) - 0.5 * W.hopping(U, psi, keep=dom.keep_inside)


def apply_R(U, psi, dom: Domains):
    """Inter-domain couplings R: only hops crossing a domain face."""
    return -0.5 * W.hopping(U, psi, keep=dom.keep_crossing)


def site_diag_inverse(F, kappa, csw, shape):
    """(1/(2 kappa) + D_cl(x))^{-1} as a 12x12 matrix per site."""
    M = np.broadcast_to(np.eye(12, dtype=np.complex128) / (2.0 * kappa), shape + (12, 12)).copy()
    if csw != 0.0:
        M = M + W.clover_matrix(F, csw)
    return np.linalg.inv(M)


def apply_site_matrix(Minv, psi):
    sh = psi.shape
    v = psi.reshape(sh[:-2] + (12,))
    return np.einsum("...ij,...j->...i", Minv, v).reshape(sh)


class BlockSolver:
    """Approximate D_Lambda^{-1} on all domains of one colour at once (they decouple).

    Even-odd reduction of Eq. 5 inside every domain:
        f~_e   = r_e - D_eo D_oo^{-1} r_o
        D~_ee  = D_ee - D_eo D_oo^{-1} D_oe        (MR on this, I_domain steps)
        delta_o = D_oo^{-1} (r_o - D_oe x_e)
    where D_ee, D_oo are the site-diagonal parts and D_eo, D_oe the domain-internal hops.
    """

    def __init__(self, U, F, kappa, csw, dom: Domains):
        self.U, self.F, self.kappa, self.csw, self.dom = U, F, kappa, csw, dom
        self.Dinv = site_diag_inverse(F, kappa, csw, U.shape[:4])
        self.even = (dom.parity == 0)[..., None, None]
        self.odd = (dom.parity == 1)[..., None, None]

    def hop_in(self, v):
        """Domain-internal hopping -1/2 D_w restricted to hops inside a domain."""
        return -0.5 * W.hopping(self.U, v, keep=self.dom.keep_inside)

    def schur(self, v_e):
        """D~_ee v_e for a vector supported on even sites."""
        t = self.odd * self.hop_in(v_e)                      # D_oe v_e
        t = apply_site_matrix(self.Dinv, t) * self.odd       # D_oo^{-1} D_oe v_e
        t = self.even * self.hop_in(t)                       # D_eo D_oo^{-1} D_oe v_e
        return self.even * diag_part(self.F, v_e, self.kappa, self.csw) - t

    def dom_dot(self, a, b, cmask):
        """Per-domain <a, b> = sum conj(a) b, broadcast back to the sites."""
        s = np.einsum("...sc,...sc->...", a.conj(), b)
        sums = np.bincount(self.dom.domain.ravel(), weights=s.real.ravel(),
                           minlength=self.dom.ndomains) \
            + 1j * np.bincount(self.dom.domain.ravel(), weights=s.imag.ravel(),
                               minlength=self.dom.ndomains)
        return sums[self.dom.domain]

    def mr(self, f_e, cmask, n_iter):
        """Minimal residual on D~_ee: x = 0, rho = f; repeat p = D~ rho,
        alpha = <p, rho>/<p, p>, x += alpha rho, rho -= alpha p.  Returns (x, rho)."""
        x = np.zeros_like(f_e)
        rho = f_e.copy()
        for _ in range(n_iter):
            p = self.schur(rho) * cmask
            num = self.dom_dot(p, rho, cmask)
            den = self.dom_dot(p, p, cmask).real
            alpha = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)[..., None, None]
            x = x + alpha * rho
            rho = rho - alpha * p
        return x, rho

    def solve(self, r, colour, n_iter):
        """delta ~ D^{-1} r on the domains of `colour` (zero elsewhere)."""
        cmask = (self.dom.colour == colour)[..., None, None].astype(np.float64)
        r = r * cmask
        r_e, r_o = r * self.even, r * self.odd
        f_e = r_e - self.even * self.hop_in(apply_site_matrix(self.Dinv, r_o) * self.odd)
        x_e, _ = self.mr(f_e * cmask, cmask, n_iter)
        d_o = apply_site_matrix(self.Dinv, r_o - self.odd * self.hop_in(x_e)) * self.odd
        return (x_e + d_o) * cmask


class ExactBlockSolver:
    """Exact D_Lambda^{-1} per domain by a dense solve (for small test lattices)."""

    def __init__(self, U, F, kappa, csw, dom: Domains):
        self.dom = dom
        shape = U.shape[:4] + (4, 3)
        n = int(np.prod(shape))
        cols = np.zeros((n, n), dtype=np.complex128)
        e = np.zeros(n, dtype=np.complex128)
        for j in range(n):
            e[:] = 0
            e[j] = 1
            cols[:, j] = apply_D(U, F, e.reshape(shape), kappa, csw, dom).ravel()
        self.D = cols
        self.shape = shape
        self.sitedom = np.repeat(dom.domain.ravel(), 12)
        self.sitecol = np.repeat(dom.colour.ravel(), 12)

    def solve(self, r, colour, n_iter=None):
        rv = r.ravel()
        out = np.zeros_like(rv)
        for d in np.unique(self.sitedom[self.sitecol == colour]):
            idx = np.nonzero(self.sitedom == d)[0]
            out[idx] = np.linalg.solve(self.D[np.ix_(idx, idx)], rv[idx])
        return out.reshape(self.shape)


def sap(U, F, f, kappa, csw, dom: Domains, i_schwarz: int, i_domain: int, solver=None):
    """Multiplicative Schwarz preconditioner M f (Table I): for s = 1..I_Schwarz, for
    colour black then white: u <- u + D_c^{-1} (f - A u)_c.  u^0 = 0."""
    if solver is None:
        solver = BlockSolver(U, F, kappa, csw, dom)
    u = np.zeros_like(f)
    for _ in range(i_schwarz):
        for colour in (0, 1):
            r = f - W.apply_A(U, u, kappa, csw, F)
            u = u + solver.solve(r, colour, i_domain)
    return u


def sap_additive(U, F, f, kappa, csw, dom: Domains, i_schwarz: int, i_domain: int, solver=None):
    """Additive Schwarz preconditioner (Sec. II-D, Eq. 4; block Jacobi): for s = 1..I_Schwarz,
    u <- u + D^{-1} (f - A u) with both colours solving from the same residual.  u^0 = 0."""
    if solver is None:
        solver = BlockSolver(U, F, kappa, csw, dom)
    u = np.zeros_like(f)
    for _ in range(i_schwarz):
        r = f - W.apply_A(U, u, kappa, csw, F)
        u = u + solver.solve(r, 0, i_domain) + solver.solve(r, 1, i_domain)
    return u
