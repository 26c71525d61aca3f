"""Pins for the oracle's FGMRES-DR (outer solver of Table I)."""
import numpy as np
import scipy.linalg as sla

from oracle.fgmres import fgmres_dr, harmonic_ritz


def mat(n, seed, shift=3.0):
    rng = np.random.default_rng(seed)
    A = shift * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    return A


def test_exact_in_n_steps():
    n = 12
    A = mat(n, 1, shift=0.5)
    b = np.random.default_rng(2).standard_normal(n) + 0j
    x, info = fgmres_dr(lambda v: A @ v, lambda v: v, b, m=n, k=0, tol=1e-13)
    assert info["iterations"] <= n
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-11 * np.linalg.norm(x)


def test_first_cycle_is_minimal_residual_over_krylov_space():
    n, m = 40, 7
    A = mat(n, 3, shift=1.0)
    b = np.random.default_rng(4).standard_normal(n) + 0j
    x, info = fgmres_dr(lambda v: A @ v, lambda v: v, b, m=m, k=0, tol=1e-30, max_cycles=1)
    K = np.zeros((n, m), dtype=complex)
    v = b.copy()
    for j in range(m):
        K[:, j] = v
        v = A @ v
    y, *_ = np.linalg.lstsq(A @ K, b, rcond=None)
    assert np.linalg.norm(x - K @ y) < 1e-10 * np.linalg.norm(x)


def test_residual_monotone_and_preconditioned():
    n = 80
    A = mat(n, 5, shift=2.0)
    D = np.diag(np.diag(A))
    b = np.random.default_rng(6).standard_normal(n) + 0j
    x, info = fgmres_dr(lambda v: A @ v, lambda v: np.linalg.solve(D, v), b, m=10, k=3, tol=1e-12)
    h = info["history"]
    assert info["true_residual"] <= 1e-12
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b)
    assert all(h[i + 1] <= h[i] * (1 + 1e-12) for i in range(min(10, len(h) - 1)))


def test_harmonic_ritz_matches_generalised_pencil():
    n, m = 60, 9
    A = mat(n, 7, shift=1.0)
    b = np.random.default_rng(8).standard_normal(n) + 0j
    rec = []
    fgmres_dr(lambda v: A @ v, lambda v: v, b, m=m, k=3, tol=1e-30, max_cycles=1, record=rec)
    Hbar = rec[0]["Hbar"]
    theta, G = harmonic_ritz(Hbar, m)
    # harmonic Ritz values: Hbar^H Hbar g = theta H_m^H g
    ref = sla.eigvals(Hbar.conj().T @ Hbar, Hbar[:m, :m].conj().T)
    ref = ref[np.argsort(np.abs(ref))]
    assert np.allclose(np.sort_complex(theta), np.sort_complex(ref), rtol=1e-9)


def test_deflated_restart_keeps_flexible_arnoldi_relation():
    """After a deflated restart A Z_k = V_{k+1} Hbar_k and V_{k+1} c_k = r still hold,
    V_{k+1} is orthonormal, and deflation does not need more steps than k = 0."""
    n, m, k = 70, 10, 4
    A = mat(n, 9, shift=1.5)
    Dg = np.diag(np.diag(A)) * 1.1
    b = np.random.default_rng(10).standard_normal(n) + 0j
    Mv = lambda v: np.linalg.solve(Dg, v)
    rec = []
    x2, info2 = fgmres_dr(lambda v: A @ v, Mv, b, m=m, k=k, tol=1e-11, record=rec)
    x0, info0 = fgmres_dr(lambda v: A @ v, Mv, b, m=m, k=0, tol=1e-11)
    assert info2["true_residual"] <= 1e-11 and info0["true_residual"] <= 1e-11
    assert info2["iterations"] <= info0["iterations"]
    restarts = [r for r in rec if "Vk" in r]
    assert restarts
    for r in restarts:
        Vk, Zk, Hk = r["Vk"].T, r["Zk"].T, r["Hk"]
        assert np.linalg.norm(A @ Zk - Vk @ Hk) < 1e-12 * np.linalg.norm(A @ Zk)
        assert np.allclose(Vk.conj().T @ Vk, np.eye(k + 1), atol=1e-13)
        # the true residual is formed by cancellation, so its error scales with the norm of b
        assert np.linalg.norm(Vk @ r["ck"] - r["r"]) < 1e-13 * np.linalg.norm(b)
