"""Oracle for the Wilson-clover operator A = (N_d + m) - 1/2 D_w + D_cl (Sec. II-B, Eq. 1).

Test infrastructure only (see the package docstring).

Readings of the paper taken here (it leaves them open):
  * gamma matrices: Euclidean, Hermitian, chiral basis with gamma_5 = g1 g2 g3 g4 =
    diag(1, 1, -1, -1), g_k = [[0, -i s_k], [i s_k, 0]] (k = x, y, z), g_t = [[0, 1], [1, 0]].
    In this basis sigma_{mu nu} is block diagonal in chirality, which gives the two
    Hermitian 6x6 clover blocks per site that Sec. II-B describes.
  * boundary conditions: periodic in x, y, z; antiperiodic in t (every hop across the
    t = L_t - 1 <-> 0 boundary carries a factor -1).
  * clover normalisation (Eq. 3 calls F_hat "a certain sum"): the standard
    Sheikholeslami-Wohlert term in this mass convention,
        D_cl(x) = -(c_sw / 32) sum_{mu != nu} gamma_mu gamma_nu (x) [Q_mu,nu(x) - Q_nu,mu(x)],
    Q_mu,nu the sum of the four plaquette leaves in the (mu, nu) plane at x.
  * mass: N_d + m = 1 / (2 kappa).
"""
from __future__ import annotations

import numpy as np

# direction mu (0..3 = x, y, z, t) -> axis of the (t, z, y, x) site block
AXIS = (3, 2, 1, 0)

_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)


def gammas() -> np.ndarray:
    """gamma_mu for mu = x, y, z, t as a (4, 4, 4) array (chiral basis, see module doc)."""
    g = [np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in (_S1, _S2, _S3)]
    g.append(np.block([[_Z2, _I2], [_I2, _Z2]]))
    return np.array(g)


def gamma5() -> np.ndarray:
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


def shift(F: np.ndarray, mu: int, step: int) -> np.ndarray:
    """F(x + step * mu_hat), periodic, for any per-site field F[t, z, y, x, ...]."""
    return np.roll(F, -step, axis=AXIS[mu])


def _t_boundary_sign(F: np.ndarray, step: int, bc_t: float) -> np.ndarray:
    """Apply the time boundary factor to a field already shifted by `step` in t.

    After shift(., t, +1) the slice t = L_t - 1 holds values from t = 0 (a wrapped hop);
    after shift(., t, -1) the slice t = 0 holds values from t = L_t - 1.
    """
    F = F.copy()
    if step > 0:
        F[-1] *= bc_t
    else:
        F[0] *= bc_t
    return F


def link_times(U_mu: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U psi)[x, s, a] = sum_b U[x, a, b] psi[x, s, b]."""
    return np.einsum("...ab,...sb->...sa", U_mu, psi)


def link_dag_times(U_mu: np.ndarray, psi: np.ndarray) -> np.ndarray:
    return np.einsum("...ba,...sb->...sa", U_mu.conj(), psi)


def spin_times(G: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(G psi)[x, s, c] = sum_t G[s, t] psi[x, t, c]."""
    return np.einsum("st,...tc->...sc", G, psi)


def hopping(U: np.ndarray, psi: np.ndarray, bc_t: float = -1.0, keep=None) -> np.ndarray:
    """Wilson hopping term of Eq. 2:

        (D_w psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                              + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ].

    `keep`, if given, is a callable keep(mu, step) -> boolean site mask (or None) that
    multiplies each hop term; the domain-restricted operators use it to drop or keep
    the hops that cross a domain face.
    """
    g = gammas()
    one = np.eye(4, dtype=np.complex128)
    out = np.zeros_like(psi)
    for mu in range(4):
        # forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
        fwd = shift(psi, mu, +1)
        if mu == 3:
            fwd = _t_boundary_sign(fwd, +1, bc_t)
        term_f = spin_times(one - g[mu], link_times(U[..., mu, :, :], fwd))
        # backward: (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)
        w = link_dag_times(U[..., mu, :, :], psi)
        bwd = shift(w, mu, -1)
        if mu == 3:
            bwd = _t_boundary_sign(bwd, -1, bc_t)
        term_b = spin_times(one + g[mu], bwd)
        if keep is not None:
            mf, mb = keep(mu, +1), keep(mu, -1)
            term_f = term_f * mf[..., None, None]
            term_b = term_b * mb[..., None, None]
        out += term_f + term_b
    return out


def _dag(M: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(M, -1, -2))


def leaves_sum(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Q_mu,nu(x): the four plaquettes in the (mu, nu) plane that start and end at x,
    each traversed in the orientation mu -> nu -> -mu -> -nu (Sec. II-B, "four-leaved
    clover").  Gauge links are periodic in every direction."""
    Um, Un = U[..., mu, :, :], U[..., nu, :, :]
    S = shift
    # leaf 1: x -> x+mu -> x+mu+nu -> x+nu -> x
    l1 = Um @ S(Un, mu, 1) @ _dag(S(Um, nu, 1)) @ _dag(Un)
    # leaf 2: x -> x+nu -> x+nu-mu -> x-mu -> x
    l2 = Un @ _dag(S(S(Um, mu, -1), nu, 1)) @ _dag(S(Un, mu, -1)) @ S(Um, mu, -1)
    # leaf 3: x -> x-mu -> x-mu-nu -> x-nu -> x
    l3 = _dag(S(Um, mu, -1)) @ _dag(S(S(Un, mu, -1), nu, -1)) @ S(S(Um, mu, -1), nu, -1) @ S(Un, nu, -1)
    # leaf 4: x -> x-nu -> x-nu+mu -> x+mu -> x
    l4 = _dag(S(Un, nu, -1)) @ S(Um, nu, -1) @ S(S(Un, nu, -1), mu, 1) @ _dag(Um)
    return l1 + l2 + l3 + l4


PLANES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def field_strength(U: np.ndarray) -> dict:
    """F_mu,nu = Q_mu,nu - Q_nu,mu for the six planes mu < nu, each Q from its own leaves."""
    return {(mu, nu): leaves_sum(U, mu, nu) - leaves_sum(U, nu, mu) for (mu, nu) in PLANES}


def clover_apply(F: dict, psi: np.ndarray, csw: float) -> np.ndarray:
    """D_cl psi with D_cl = -(c_sw/32) sum_{mu != nu} gamma_mu gamma_nu (x) F_mu,nu.

    The sum over ordered pairs is written out as the pairs (mu, nu) and (nu, mu) for
    mu < nu, using F_nu,mu = Q_nu,mu - Q_mu,nu = -F_mu,nu.
    """
    g = gammas()
    out = np.zeros_like(psi)
    for (mu, nu), Fmn in F.items():
        spin = g[mu] @ g[nu] - g[nu] @ g[mu]
        out += spin_times(spin, link_times(Fmn, psi))
    return -(csw / 32.0) * out


def clover_matrix(F: dict, csw: float) -> np.ndarray:
    """The 12x12 matrix of D_cl at every site, index (spin, colour) -> 3*spin + colour."""
    g = gammas()
    shape = next(iter(F.values())).shape[:-2]
    M = np.zeros(shape + (12, 12), dtype=np.complex128)
    for (mu, nu), Fmn in F.items():
        spin = g[mu] @ g[nu] - g[nu] @ g[mu]
        M += np.einsum("st,...ab->...satb", spin, Fmn).reshape(shape + (12, 12))
    return -(csw / 32.0) * M


def apply_A(U: np.ndarray, psi: np.ndarray, kappa: float, csw: float, F: dict | None = None,
            bc_t: float = -1.0) -> np.ndarray:
    """A psi = (1/(2 kappa)) psi - 1/2 D_w psi + D_cl psi  (Eq. 1 with N_d + m = 1/(2 kappa))."""
    if F is None and csw != 0.0:
        F = field_strength(U)
    out = psi / (2.0 * kappa) - 0.5 * hopping(U, psi, bc_t)
    if csw != 0.0:
        out = out + clover_apply(F, psi, csw)
    return out


# ----------------------------------------------------------------------------------
# Per-site evaluation for sampled checks on lattices too large for the vectorised path.
# Explicit neighbour coordinates; same definitions as above, one site at a time.
# ----------------------------------------------------------------------------------

def _site(coord, dims):
    x, y, z, t = coord
    Lx, Ly, Lz, Lt = dims
    return (t % Lt, z % Lz, y % Ly, x % Lx)


def _step(coord, mu, s):
    c = list(coord)
    c[mu] += s
    return tuple(c)


def apply_A_at(U: np.ndarray, psi: np.ndarray, kappa: float, csw: float, coords,
               bc_t: float = -1.0) -> np.ndarray:
    """(A psi)(x) for each x = (x, y, z, t) in coords; returns (n, 4, 3)."""
    Lt, Lz, Ly, Lx = psi.shape[:4]
    dims = (Lx, Ly, Lz, Lt)
    g = gammas()
    one = np.eye(4, dtype=np.complex128)

    def link(c, mu):
        return U[_site(c, dims) + (mu,)]

    def sign(c_from, c_to):
        # a hop whose time coordinate wraps picks up bc_t
        t0, t1 = c_from[3], c_to[3]
        return bc_t if (t1 >= Lt or t1 < 0) and t0 != t1 else 1.0

    out = []
    for c in coords:
        c = tuple(int(v) for v in c)
        v = psi[_site(c, dims)] / (2 * kappa)
        hop = np.zeros((4, 3), dtype=np.complex128)
        for mu in range(4):
            cf, cb = _step(c, mu, 1), _step(c, mu, -1)
            pf = psi[_site(cf, dims)] * sign(c, cf)
            hop += (one - g[mu]) @ (link(c, mu) @ pf.T).T
            pb = psi[_site(cb, dims)] * sign(c, cb)
            hop += (one + g[mu]) @ (link(cb, mu).conj().T @ pb.T).T
        v = v - 0.5 * hop
        if csw != 0.0:
            acc = np.zeros((4, 3), dtype=np.complex128)
            for mu in range(4):
                for nu in range(4):
                    if mu == nu:
                        continue
                    Q = _leaves_at(link, c, mu, nu)
                    Qr = _leaves_at(link, c, nu, mu)
                    acc += (g[mu] @ g[nu]) @ ((Q - Qr) @ psi[_site(c, dims)].T).T
            v = v - (csw / 32.0) * acc
        out.append(v)
    return np.array(out)


def _leaves_at(link, c, mu, nu):
    S = _step
    d = lambda M: M.conj().T
    l1 = link(c, mu) @ link(S(c, mu, 1), nu) @ d(link(S(c, nu, 1), mu)) @ d(link(c, nu))
    l2 = link(c, nu) @ d(link(S(S(c, nu, 1), mu, -1), mu)) @ d(link(S(c, mu, -1), nu)) @ link(S(c, mu, -1), mu)
    l3 = d(link(S(c, mu, -1), mu)) @ d(link(S(S(c, mu, -1), nu, -1), nu)) @ link(S(S(c, mu, -1), nu, -1), mu) @ link(S(c, nu, -1), nu)
    l4 = d(link(S(c, nu, -1), nu)) @ link(S(c, nu, -1), mu) @ link(S(S(c, nu, -1), mu, 1), nu) @ d(link(c, mu))
    return l1 + l2 + l3 + l4
