"""The deflated restart's small dense step as dd_solve runs it on the device (one warp,
FP64): against the oracle's harmonic Ritz pairs (Sec. II-C, GMRES-DR) and against the same
team code run on the host, on the Hessenberg matrices of three FGMRES-DR cycles (the later
ones with the dense leading block a deflated restart leaves), including the basis size and
deflation count of the 32^3x64 solve (m = 40, k = 8)."""
import numpy as np
import pytest

from oracle.fgmres import fgmres_dr, harmonic_ritz
from paper_1412_2629_gb300 import dd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m,k,seed", [(60, 10, 4, 3), (160, 40, 8, 4)])
def test_device_deflation_matches_oracle_and_host(n, m, k, seed):
    rng = np.random.default_rng(seed)
    A = 1.2 * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 0j
    rec = []
    fgmres_dr(lambda v: A @ v, lambda v: v, b, m=m, k=k, tol=1e-30, max_cycles=3, record=rec)
    for r in rec:
        Hbar, c, y = r["Hbar"], r["c"], r["y"]
        mm = Hbar.shape[1]
        P, Hn, cn, th, ms = dd.dd_deflate_device(Hbar, c, y, k)
        print(f"m {mm} k {k}: device deflation {ms:.3f} ms")
        theta, G = harmonic_ritz(Hbar, mm)
        # the k kept values FP64 accurate, the others FP32 estimates (nearest exact value)
        scale = np.abs(Hbar).max()
        for i, t in enumerate(th):
            assert np.abs(theta - t).min() <= (1e-10 * abs(t) + 1e-12 * scale if i < k else 1e-4 * scale)
        assert np.allclose(P.conj().T @ P, np.eye(k + 1), atol=1e-12)
        Gk = np.vstack([G[:, :k], np.zeros((1, k))])
        proj = P[:, :k] @ (P[:, :k].conj().T @ Gk)
        assert np.linalg.norm(proj - Gk) < 1e-9 * np.linalg.norm(Gk)
        assert np.allclose(P @ cn, c - Hbar @ y, atol=1e-12 * np.linalg.norm(c))
        assert np.allclose(Hn, P.conj().T @ Hbar @ P[:mm, :k], atol=1e-12 * np.linalg.norm(Hbar))
        # the host run of the same code: same Ritz values, same subspace (each eigenvector is
        # fixed only up to a phase, which rounding may settle differently)
        Ph, Hnh, cnh, thh = dd.dd_deflate_host(Hbar, c, y, k)
        assert np.allclose(th[:k], thh[:k], rtol=1e-9, atol=1e-12)
        assert np.linalg.norm(P @ P.conj().T - Ph @ Ph.conj().T) <= 1e-8 * (k + 1)
