"""GPU parity of the two-level multigrid with the Schwarz smoother (related work, Sec. V)
against the oracle (oracle/mg.py) on the same seeded inputs.

Bars:
  * restriction / prolongation: FP32 fields and interpolation, sums of a few thousand
    terms per aggregate: 1e-5 relative L2 (u_32 = 6e-8 times the growth of the FP32
    Gram-Schmidt, which the oracle's QR does in FP64);
  * coarse operator: built in FP32 from FP32 links and clover: 1e-4 relative;
  * coarse solve: GMRES(32) x 3 cycles in FP32 on at most 256 unknowns reaches the FP32
    floor of the coarse system: 1e-4 relative against the dense FP64 solve;
  * one application of the preconditioner (coarse solve plus one FP32-storage Schwarz
    cycle, itself held to 1e-5 against the oracle): 2e-4 relative.
The lattices have 2 domains per direction (the +mu and -mu neighbours of a domain
coincide, two coarse blocks act on the same site) and 4 domains in x (distinct
neighbours)."""
import numpy as np
import pytest
import torch

import synth
from oracle import dd as DD
from oracle import mg as MG
from oracle import solve as OS
from oracle import wilson as W
from paper_1412_2629_gb300 import dd

from gpu_helpers import ctx_for, dev, gauge, host, rel

pytestmark = pytest.mark.gpu

KAPPA, CSW = 0.124, 1.3
CASES = [((8, 8, 8, 8), (4, 4, 4, 4), 21), ((16, 8, 8, 8), (4, 4, 4, 4), 22)]
NTV = 4


def _coarse_shape(dims, dom):
    return tuple(L // b for L, b in zip(dims, dom))[::-1] + (2, NTV)


def _tv(dims, seed):
    return [synth.gaussian_source(dims, seed + 100 + k) for k in range(NTV)]


def _setup(dims, dom, seed, setup_iters=0, i_schwarz=1, coarse_m=32, cycles=3, mode=0):
    U = gauge(dims, 0.5, seed, ape=2)
    c = ctx_for(dims, dom, U, KAPPA, CSW)
    tv = _tv(dims, seed)
    t = torch.stack([dev(v) for v in tv]).contiguous()
    c.dd_mg_setup(t, NTV, dd.DD_DEVICE, setup_iters=setup_iters, coarse_m=coarse_m, coarse_cycles=cycles,
                  i_schwarz=i_schwarz, i_domain=4, storage_prec=dd.DD_PREC_FP32, threads_per_site=2,
                  setup_mode=mode)
    return U, c, tv


def _internal(c, psi):
    src = dev(psi, torch.float32)
    buf = torch.empty_like(src)
    c.dd_pack_spinor(src, dd.DD_PREC_FP32, buf, dd.DD_PREC_FP32)
    return buf


def _canonical(c, buf):
    out = torch.empty_like(buf)
    c.dd_unpack_spinor(buf, dd.DD_PREC_FP32, out, dd.DD_PREC_FP32)
    return host(out)


def _cvec(x):
    return torch.view_as_real(torch.from_numpy(np.ascontiguousarray(x.ravel()).astype(np.complex64))).cuda().contiguous()


def _chost(t):
    a = t.cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
def test_restrict_prolong_match_oracle(case):
    dims, dom, seed = case
    U, c, tv = _setup(dims, dom, seed)
    agg = MG.Aggregates(dims, dom)
    P = MG.interpolation(tv, agg)
    r = synth.gaussian_source(dims, seed + 50)
    rc = torch.empty(agg.n * 2 * NTV, 2, dtype=torch.float32, device="cuda")
    c.dd_mg_restrict(_internal(c, r), rc)
    assert rel(_chost(rc), MG.restrict(P, agg, r).ravel()) <= 1e-5
    rng = np.random.default_rng(seed)
    shape = _coarse_shape(dims, dom)
    e = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    out = torch.empty(c.dd_spinor_bytes(dd.DD_PREC_FP32, dd.DD_LAYOUT_INTERNAL) // 4, dtype=torch.float32,
                      device="cuda")
    c.dd_mg_prolong(_cvec(e), out)
    got = _canonical(c, out.view(dims[3], dims[2], dims[1], dims[0], 4, 3, 2))
    assert rel(got, MG.prolong(P, agg, e)) <= 1e-5


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
def test_coarse_operator_and_solve_match_oracle(case):
    dims, dom, seed = case
    U, c, tv = _setup(dims, dom, seed)
    agg = MG.Aggregates(dims, dom)
    P = MG.interpolation(tv, agg)
    Dc = MG.coarse_matrix(U, KAPPA, CSW, P, agg)
    rng = np.random.default_rng(seed + 1)
    n = Dc.shape[0]
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = torch.empty(n, 2, dtype=torch.float32, device="cuda")
    c.dd_mg_coarse_apply(_cvec(x), y)
    assert rel(_chost(y), Dc @ x) <= 1e-4
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    xs = torch.empty(n, 2, dtype=torch.float32, device="cuda")
    c.dd_mg_coarse_solve(_cvec(b), xs)
    assert rel(_chost(xs), np.linalg.solve(Dc, b)) <= 1e-4


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
def test_precondition_matches_oracle(case):
    dims, dom, seed = case
    U, c, tv = _setup(dims, dom, seed)
    agg = MG.Aggregates(dims, dom)
    doms = DD.Domains(dims, dom)
    F = W.field_strength(U)
    P = MG.interpolation(tv, agg)
    Dc = MG.coarse_matrix(U, KAPPA, CSW, P, agg, F)
    b = synth.gaussian_source(dims, seed + 60)
    ref = MG.two_level(U, KAPPA, CSW, P, agg, Dc, b, doms, 1, 4, F)
    src = dev(b, torch.float32)
    out = torch.empty_like(src)
    c.dd_mg_precondition(src, out, dd.DD_LAYOUT_CANONICAL)
    assert rel(host(out), ref) <= 2e-4


@pytest.mark.parametrize("mode", [0, 1], ids=["inverse", "nullspace"])
def test_smoothed_setup_matches_oracle(mode):
    """Two smoothing steps per test vector before the interpolation is built (FP32 storage;
    mode 0: v <- M_sap v, mode 1: v <- v - M_sap A v): the GPU's interpolation and coarse
    operator act like the oracle's within 1e-3 (the smoothed vectors agree to the Schwarz
    bar of 1e-5; the Gram-Schmidt of vectors that the smoothing has turned towards the same
    low modes amplifies that difference)."""
    dims, dom, seed = CASES[0]
    U, c, tv = _setup(dims, dom, seed, setup_iters=2, mode=mode)
    agg = MG.Aggregates(dims, dom)
    doms = DD.Domains(dims, dom)
    F = W.field_strength(U)
    P, Dc = MG.setup(U, KAPPA, CSW, tv, agg, 2, doms, 1, 4, F, mode=("inverse", "nullspace")[mode])
    r = synth.gaussian_source(dims, seed + 70)
    rc = torch.empty(agg.n * 2 * NTV, 2, dtype=torch.float32, device="cuda")
    c.dd_mg_restrict(_internal(c, r), rc)
    assert rel(_chost(rc), MG.restrict(P, agg, r).ravel()) <= 1e-3
    rng = np.random.default_rng(seed + 2)
    x = rng.standard_normal(Dc.shape[0]) + 1j * rng.standard_normal(Dc.shape[0])
    y = torch.empty(Dc.shape[0], 2, dtype=torch.float32, device="cuda")
    c.dd_mg_coarse_apply(_cvec(x), y)
    assert rel(_chost(y), Dc @ x) <= 1e-3


def test_solve_mg_true_residual_and_fewer_iterations():
    """FGMRES-DR with the two-level preconditioner reaches 1e-10 (true residual recomputed
    by the oracle) in fewer outer steps than with the Schwarz method alone."""
    dims, dom = (16, 8, 8, 8), (4, 4, 4, 4)
    U = gauge(dims, 0.5, 23, ape=2)
    kappa = 0.1265
    c = ctx_for(dims, dom, U, kappa, CSW)
    tv = torch.stack([dev(synth.gaussian_source(dims, 300 + k)) for k in range(8)]).contiguous()
    c.dd_mg_setup(tv, 8, dd.DD_DEVICE, setup_iters=3, coarse_m=24, coarse_cycles=1, i_schwarz=2, i_domain=4,
                  storage_prec=dd.DD_PREC_FP16)
    f = synth.gaussian_source(dims, 24)
    x = np.zeros_like(f)
    xv = torch.view_as_real(torch.from_numpy(x)).contiguous()
    fv = torch.view_as_real(torch.from_numpy(f)).contiguous()
    info = c.dd_solve_mg(fv, xv, where=dd.DD_HOST, tol=1e-10, m=16, k=4, max_iter=2000)
    x = xv.numpy()[..., 0] + 1j * xv.numpy()[..., 1]
    assert OS.true_residual(U, x, f, kappa, CSW) <= 1.05e-10
    x2 = torch.zeros_like(fv)
    info_sap = c.dd_solve(fv, x2, where=dd.DD_HOST, tol=1e-10, m=16, k=4, max_iter=4000, i_schwarz=2, i_domain=4,
                          storage_prec=dd.DD_PREC_FP16)
    assert info.iterations < info_sap.iterations
    # a second solve on the same context replays the captured steps: same result bit for bit
    x3 = torch.zeros_like(fv)
    info3 = c.dd_solve_mg(fv, x3, where=dd.DD_HOST, tol=1e-10, m=16, k=4, max_iter=2000)
    assert info3.iterations == info.iterations
    assert torch.equal(x3, xv)


def test_mg_setup_rejects_bad_parameters():
    dims, dom = (8, 8, 8, 8), (4, 4, 4, 4)
    U = gauge(dims, 0.5, 25)
    c = ctx_for(dims, dom, U, KAPPA, CSW)
    tv = torch.zeros(17, *dims[::-1], 4, 3, 2, dtype=torch.float64, device="cuda")
    for kw in (dict(n_tv=0), dict(n_tv=17), dict(n_tv=2, coarse_m=0), dict(n_tv=2, coarse_cycles=0),
               dict(n_tv=2, setup_mode=2)):
        n = kw.pop("n_tv")
        with pytest.raises(dd.DDError) as e:
            c.dd_mg_setup(tv, n, dd.DD_DEVICE, **kw)
        assert e.value.status == dd.DD_ERR_INVALID
    # zero test vectors: no basis on any aggregate
    with pytest.raises(dd.DDError) as e:
        c.dd_mg_setup(tv, 2, dd.DD_DEVICE, setup_iters=0)
    assert e.value.status == dd.DD_ERR_NONFINITE
    src = torch.zeros(*dims[::-1], 4, 3, 2, dtype=torch.float32, device="cuda")
    with pytest.raises(dd.DDError):
        c.dd_mg_precondition(src, torch.empty_like(src))


def test_coarse_operator_odd_test_vector_count():
    """Three test vectors (six coarse unknowns per domain: the row-length-at-run-time form of
    the coarse operator) against the oracle's D_c."""
    dims, dom, seed = CASES[1]
    U = gauge(dims, 0.5, seed, ape=2)
    c = ctx_for(dims, dom, U, KAPPA, CSW)
    tv = [synth.gaussian_source(dims, seed + 200 + k) for k in range(3)]
    c.dd_mg_setup(torch.stack([dev(v) for v in tv]).contiguous(), 3, dd.DD_DEVICE, setup_iters=0, coarse_m=16,
                  coarse_cycles=2, i_schwarz=1, i_domain=4, storage_prec=dd.DD_PREC_FP32, threads_per_site=2)
    agg = MG.Aggregates(dims, dom)
    Dc = MG.coarse_matrix(U, KAPPA, CSW, MG.interpolation(tv, agg), agg)
    rng = np.random.default_rng(seed + 3)
    x = rng.standard_normal(Dc.shape[0]) + 1j * rng.standard_normal(Dc.shape[0])
    y = torch.empty(Dc.shape[0], 2, dtype=torch.float32, device="cuda")
    c.dd_mg_coarse_apply(_cvec(x), y)
    assert rel(_chost(y), Dc @ x) <= 1e-4
