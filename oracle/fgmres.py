"""Oracle for the outer solver: flexible GMRES with deflated restarts (Table I, Sec. II-B).

Test infrastructure only (see the package docstring).

The paper only cites the method (Frommer et al.); the steps follow Morgan's GMRES-DR
with flexible right preconditioning:
  * first cycle: flexible GMRES(m): v_1 = r / |r|, z_j = M v_j, w = A z_j, Gram-Schmidt of
    w against v_1..v_j gives column j of the (m+1) x m Hessenberg matrix Hbar, and
    A Z_m = V_{m+1} Hbar.  y minimises | c - Hbar y | (c = |r| e_1), x += Z_m y.
  * restart with k > 0: the harmonic Ritz pairs of Hbar solve
        (H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^H) g = theta g,
    the k of smallest |theta| are kept (ties broken by the order of a stable sort on
    |theta|).  P_{k+1} is an orthonormal basis of [g_1 .. g_k ; 0] followed by the
    least-squares residual vector c - Hbar y; then V <- V_{m+1} P_{k+1}, Z <- Z_m P_k,
    Hbar <- P_{k+1}^H Hbar P_k, c <- P_{k+1}^H (c - Hbar y), and Arnoldi resumes at
    step k + 1 orthogonalising against all k + 1 vectors.
  * k = 0 is restarted flexible GMRES(m) from the true residual.
  * a cycle ends after m steps or when the least-squares residual drops below tol |b|;
    the true residual b - A x is then formed and decides convergence.
The Gram-Schmidt step is modified Gram-Schmidt applied twice (full reorthogonalisation),
all in FP64.
"""
from __future__ import annotations

import numpy as np


def _orth(basis, w):
    h = np.zeros(len(basis), dtype=np.complex128)
    for _ in range(2):
        for i, v in enumerate(basis):
            c = np.vdot(v, w)
            h[i] += c
            w = w - c * v
    return h, w


def harmonic_ritz(Hbar: np.ndarray, m: int):
    """Eigenpairs of H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^H, sorted by |theta| ascending."""
    Hm = Hbar[:m, :m]
    em = np.zeros(m, dtype=np.complex128)
    em[-1] = 1.0
    f = np.linalg.solve(Hm.conj().T, em)
    G = Hm + abs(Hbar[m, m - 1]) ** 2 * np.outer(f, em)
    theta, vec = np.linalg.eig(G)
    order = np.argsort(np.abs(theta), kind="stable")
    return theta[order], vec[:, order]


def fgmres_dr(A, M, b, m, k, tol=1e-10, x0=None, max_cycles=200, record=None):
    """Solve A x = b with right preconditioner M.  A, M: callables on flat complex vectors.

    Returns (x, info) with info = dict(cycles, iterations, true_residual, history).
    `record`, if a list, receives per-cycle dicts (Hbar, c, theta) for tests.
    """
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - A(x)
    beta = np.linalg.norm(r)
    hist = [beta / nb]
    if beta <= tol * nb:
        return x, dict(cycles=0, iterations=0, true_residual=beta / nb, history=hist)
    V = [r / beta]
    Z = []
    Hbar = np.zeros((m + 1, m), dtype=np.complex128)
    c = np.zeros(m + 1, dtype=np.complex128)
    c[0] = beta
    j0 = 0
    iters = 0
    for cycle in range(max_cycles):
        mm = m
        for j in range(j0, m):
            z = M(V[j])
            w = A(z)
            h, w = _orth(V, w)
            Hbar[:j + 1, j] = h
            Hbar[j + 1, j] = np.linalg.norm(w)
            V.append(w / Hbar[j + 1, j])
            Z.append(z)
            iters += 1
            y, *_ = np.linalg.lstsq(Hbar[:j + 2, :j + 1], c[:j + 2], rcond=None)
            res = np.linalg.norm(c[:j + 2] - Hbar[:j + 2, :j + 1] @ y)
            hist.append(res / nb)
            if res <= tol * nb:
                mm = j + 1
                break
        Hc = Hbar[:mm + 1, :mm].copy()
        y, *_ = np.linalg.lstsq(Hc, c[:mm + 1], rcond=None)
        x = x + sum(y[i] * Z[i] for i in range(mm))
        r = b - A(x)
        rn = np.linalg.norm(r)
        if record is not None:
            record.append(dict(Hbar=Hc, c=c[:mm + 1].copy(), y=y))
        if rn <= tol * nb:
            return x, dict(cycles=cycle + 1, iterations=iters, true_residual=rn / nb, history=hist)
        if k == 0 or mm < m or k >= mm:
            V = [r / rn]
            Z = []
            Hbar = np.zeros((m + 1, m), dtype=np.complex128)
            c = np.zeros(m + 1, dtype=np.complex128)
            c[0] = rn
            j0 = 0
            continue
        # deflated restart
        theta, G = harmonic_ritz(Hc, mm)
        cls = c[:mm + 1] - Hc @ y
        P = np.zeros((mm + 1, k + 1), dtype=np.complex128)
        Gk = np.vstack([G[:, :k], np.zeros((1, k))])
        Q, _ = np.linalg.qr(Gk)
        P[:, :k] = Q
        q = cls - Q @ (Q.conj().T @ cls)
        q = q - Q @ (Q.conj().T @ q)
        P[:, k] = q / np.linalg.norm(q)
        if record is not None:
            record[-1].update(theta=theta, P=P)
        Vm = np.array(V[:mm + 1])
        Zm = np.array(Z[:mm])
        V = list(P.T @ Vm)                       # V_{k+1} = V_{m+1} P_{k+1}
        Z = list(P[:mm, :k].T @ Zm)              # Z_k = Z_m P_k
        Hn = P.conj().T @ Hc @ P[:mm, :k]        # (k+1) x k
        Hbar = np.zeros((m + 1, m), dtype=np.complex128)
        Hbar[:k + 1, :k] = Hn
        c = np.zeros(m + 1, dtype=np.complex128)
        c[:k + 1] = P.conj().T @ cls
        if record is not None:
            record[-1].update(Vk=np.array(V), Zk=np.array(Z), Hk=Hn.copy(), ck=c[:k + 1].copy(), r=r)
        j0 = k
    return x, dict(cycles=max_cycles, iterations=iters, true_residual=rn / nb, history=hist)
