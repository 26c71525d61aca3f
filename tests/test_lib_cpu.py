"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/dd.h declares, and its pure host functions match the paper's worked values
and the oracle.  No compute call touches a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dd.h")
GOLD = os.path.join(ROOT, "tests", "golden", "load_model_table3.txt")


@pytest.fixture(scope="module")
def ddmod():
    from paper_1412_2629_gb300 import build as B
    B.build()
    from paper_1412_2629_gb300 import dd
    return dd


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dd_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("dd_load_gauge", "dd_build_clover", "dd_apply_D", "dd_sap_precondition", "dd_solve"):
        assert want in names


def test_library_exports_every_declared_symbol(ddmod):
    L = ctypes.CDLL(ddmod.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_load_model_matches_paper_values(ddmod):
    """dd_load_model is the GPU analogue of Eq. 7 (slots = resident CTAs instead of
    cores); with slots = 60 it must reproduce the paper's load column."""
    for line in open(GOLD):
        if not line.strip() or line.startswith("#"):
            continue
        kind, lat, nodes, ndom, pct = line.split()
        if kind in ("table", "text"):
            assert round(100 * ddmod.dd_load_model(int(ndom), 60)) == int(pct)
    assert ddmod.dd_load_model(2048, 152) == pytest.approx(2048 / (152 * 14))
    assert ddmod.dd_load_model(0, 152) == 0.0


def _check_ritz_values(th, theta, k, Hbar):
    """The k kept harmonic Ritz values (smallest modulus) are FP64 accurate, the others FP32
    estimates: each returned value is matched to the nearest exact one."""
    order = np.argsort(np.abs(theta), kind="stable")
    assert np.allclose(np.abs(th[:k]), np.abs(theta[order[:k]]), rtol=1e-10)
    scale = np.abs(Hbar).max()
    for i, t in enumerate(th):
        err = np.abs(theta - t).min()
        assert err <= (1e-10 * abs(t) + 1e-12 * scale if i < k else 1e-4 * scale)


@pytest.mark.parametrize("n,m,k,seed", [(60, 10, 4, 3), (160, 40, 8, 4), (120, 32, 8, 5), (90, 16, 6, 6)])
def test_host_deflation_matches_oracle(ddmod, n, m, k, seed):
    """The deflated restart's small dense step (the same team code the solver runs as one
    warp on the device, here with a team of one) against the oracle's harmonic Ritz pairs
    (Sec. II-C, GMRES-DR) on the Hessenberg matrices of a first FGMRES cycle, including the
    basis size and deflation count of the 32^3x64 solve (m = 40, k = 8)."""
    from oracle.fgmres import fgmres_dr, harmonic_ritz
    rng = np.random.default_rng(seed)
    A = 1.2 * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 0j
    rec = []
    # three cycles: after a deflated restart the leading (k+1) x k block of Hbar is dense
    fgmres_dr(lambda v: A @ v, lambda v: v, b, m=m, k=k, tol=1e-30, max_cycles=3, record=rec)
    assert len(rec) == 3
    for r in rec:
        Hbar, c, y = r["Hbar"], r["c"], r["y"]
        mm = Hbar.shape[1]
        P, Hn, cn, th = ddmod.dd_deflate_host(Hbar, c, y, k)
        theta, G = harmonic_ritz(Hbar, mm)
        _check_ritz_values(th, theta, k, Hbar)
        # P is orthonormal, spans the k kept harmonic Ritz vectors and the LS residual
        assert np.allclose(P.conj().T @ P, np.eye(k + 1), atol=1e-12)
        Gk = np.vstack([G[:, :k], np.zeros((1, k))])
        proj = P[:, :k] @ (P[:, :k].conj().T @ Gk)
        assert np.linalg.norm(proj - Gk) < 1e-9 * np.linalg.norm(Gk)
        cls = c - Hbar @ y
        assert np.allclose(P @ cn, cls, atol=1e-12 * np.linalg.norm(c))
        assert np.allclose(Hn, P.conj().T @ Hbar @ P[:mm, :k], atol=1e-12 * np.linalg.norm(Hbar))


def _create(ddmod, dims, dom):
    L = ddmod.lib()
    h = ctypes.c_void_p()
    s = L.dd_create(ctypes.byref(h), (ctypes.c_int * 4)(*dims), (ctypes.c_int * 4)(*dom), 1, None)
    if s == 0:
        L.dd_destroy(h)
    return s


@pytest.mark.parametrize("dims,dom", [
    ((16, 8, 8, 8), (8, 4, 4, 3)),     # b_mu not a power of two (and L / b not whole)
    ((12, 8, 8, 8), (4, 4, 4, 4)),     # 3 domains in x: the two colours would not alternate
    ((8, 8, 8, 8), (8, 4, 4, 4)),      # one domain in x: a hop would wrap into its own domain
    ((8, 8, 8, 8), (2, 2, 2, 2)),      # 16 sites per domain: below a warp pair
    ((32, 32, 32, 32), (8, 8, 4, 4)),  # 1024 sites per domain: above the CTA's threads
    ((0, 8, 8, 8), (4, 4, 4, 4)),
], ids=["b3", "odd_count", "one_domain", "tiny_domain", "huge_domain", "zero_extent"])
def test_create_rejects_disallowed_shapes(ddmod, dims, dom):
    """Domain constraints of the C ABI (Sec. II-D): b_mu a power of two, L_mu / b_mu even
    and at least 2 (consistent two-colouring under periodic wrap), 64..512 sites per
    domain.  Checked before any device call, so this holds without a GPU."""
    assert _create(ddmod, dims, dom) == ddmod.DD_ERR_DIMS


def test_null_arguments_are_invalid_not_fatal(ddmod):
    L = ddmod.lib()
    assert L.dd_create(None, (ctypes.c_int * 4)(8, 8, 8, 8), (ctypes.c_int * 4)(4, 4, 4, 4), 1, None) == \
        ddmod.DD_ERR_INVALID
    assert L.dd_destroy(None) == ddmod.DD_ERR_INVALID
    assert L.dd_load_gauge(None, None, 0) == ddmod.DD_ERR_INVALID
    assert L.dd_solve(None, None, None, 1, 0, None, None) == ddmod.DD_ERR_INVALID
    assert L.dd_mg_setup(None, None, 0, None, None) == ddmod.DD_ERR_INVALID
    assert L.dd_mg_restrict(None, None, None) == ddmod.DD_ERR_INVALID
    assert L.dd_mg_prolong(None, None, None) == ddmod.DD_ERR_INVALID
    assert L.dd_mg_coarse_apply(None, None, None) == ddmod.DD_ERR_INVALID
    assert L.dd_mg_coarse_solve(None, None, None) == ddmod.DD_ERR_INVALID
    assert L.dd_mg_precondition(None, None, None, 0) == ddmod.DD_ERR_INVALID
    assert L.dd_solve_mg(None, None, None, 0, None, None) == ddmod.DD_ERR_INVALID


def test_host_deflation_rejects_bad_sizes(ddmod):
    z = np.zeros(64 * 64 * 2)
    for m, k in ((0, 0), (8, 0), (8, 8), (64, 4)):
        assert ddmod.lib().dd_deflate_host(m, k, *([z.ctypes.data] * 7)) == ddmod.DD_ERR_INVALID
