"""End-to-end: dd_solve's solution, checked by the oracle in FP64 (true residual) and
against the oracle's own SAP-FGMRES-DR solution and a sparse direct solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl
import torch

import synth
from oracle import dense as DN
from oracle import solve as S
from oracle import wilson as W
from paper_1412_2629_gb300 import dd

from gpu_helpers import ctx_for, gauge, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [dd.DD_PREC_FP16, dd.DD_PREC_FP32, dd.DD_PREC_FP16_H2], ids=["mixed", "fp32", "half2"])
def test_solve_8x4_workload(prec):
    w = synth.WORKLOADS["8^4"]
    U = synth.make_gauge(w).numpy()
    f = synth.make_sources(w)[0]
    c = ctx_for(w.dims, w.domain, U, w.kappa, w.csw)
    x = np.zeros_like(f)
    info = c.dd_solve(f, x, tol=w.tol, m=w.m, k=w.k, i_schwarz=w.i_schwarz, i_domain=w.i_domain, storage_prec=prec)
    assert S.true_residual(U, x, f, w.kappa, w.csw) <= 1e-10
    assert info.true_rel_residual <= 1e-10
    xo, _ = S.solve(U, f, w.kappa, w.csw, w.domain, w.i_schwarz, w.i_domain, w.m, w.k, tol=1e-12)
    assert rel(x, xo) <= 1e-8


@pytest.mark.parametrize("basis16", [0, 1], ids=["fp32basis", "fp16basis"])
def test_solve_matches_sparse_direct_with_deflation(basis16):
    dims, dom = (8, 8, 4, 4), (4, 4, 2, 2)
    U = gauge(dims, 0.5, 21, ape=2)
    f = synth.gaussian_source(dims, 22)
    kappa, csw = 0.1390, 1.5
    c = ctx_for(dims, dom, U, kappa, csw)
    x = np.zeros_like(f)
    info = c.dd_solve(f, x, tol=1e-10, m=6, k=3, i_schwarz=2, i_domain=2, storage_prec=dd.DD_PREC_FP16,
                      basis_fp16=basis16)
    A = DN.assemble_A(U, kappa, csw).tocsc()
    xl = spl.spsolve(A, f.ravel()).reshape(f.shape)
    assert S.true_residual(U, x, f, kappa, csw) <= 1e-10
    cond_bound = 1e-10 * 1e3
    assert rel(x, xl) <= cond_bound
    assert info.restarts >= 1


def test_initial_guess_and_zero_source():
    w = synth.WORKLOADS["8^4"]
    U = synth.make_gauge(w).numpy()
    f = synth.make_sources(w)[0]
    c = ctx_for(w.dims, w.domain, U, w.kappa, w.csw)
    x = np.zeros_like(f)
    c.dd_solve(f, x, tol=1e-10, m=16, k=0, i_schwarz=16, i_domain=4)
    x2 = x.copy()
    info = c.dd_solve(f, x2, tol=1e-10, m=16, k=0, i_schwarz=16, i_domain=4)
    assert info.iterations == 0 and np.array_equal(x2, x)
    z = np.zeros_like(f)
    xz = np.ones_like(f)
    c.dd_solve(z, xz, tol=1e-10, m=16, k=0, i_schwarz=16, i_domain=4)
    assert np.abs(xz).max() == 0


def test_graph_replay_matches_direct_launches(monkeypatch):
    """Arnoldi steps replayed from captured CUDA graphs (from the second occurrence of a
    step on) give bit-for-bit the solution of direct launches (DD_NO_GRAPHS=1)."""
    dims, dom = (16, 8, 8, 8), (8, 4, 4, 4)
    U = gauge(dims, 0.5, 31, ape=2)
    f = synth.gaussian_source(dims, 32)
    kw = dict(tol=1e-10, m=8, k=2, i_schwarz=2, i_domain=3, storage_prec=dd.DD_PREC_FP16)
    c = ctx_for(dims, dom, U, 0.1250, 1.5)
    xs = []
    for _ in range(3):
        x = np.zeros_like(f)
        info = c.dd_solve(f, x, **kw)
        xs.append(x)
    assert info.restarts >= 1
    assert np.array_equal(xs[0], xs[1]) and np.array_equal(xs[1], xs[2])
    monkeypatch.setenv("DD_NO_GRAPHS", "1")
    c2 = ctx_for(dims, dom, U, 0.1250, 1.5)
    xd = np.zeros_like(f)
    c2.dd_solve(f, xd, **kw)
    assert np.array_equal(xd, xs[0])
    assert S.true_residual(U, xd, f, 0.1250, 1.5) <= 1e-10


@pytest.fixture(scope="module")
def bench_lattice():
    """The 32^3x64 workload on the GPU, and the oracle's field strength of its links."""
    w = synth.WORKLOADS["32^3x64"]
    Ud = synth.make_gauge(w, device="cuda")
    c = ctx_for(w.dims, w.domain, Ud, w.kappa, w.csw)
    U = Ud.cpu().numpy()
    del Ud
    return w, c, U, W.field_strength(U), synth.make_sources(w)[0]


@pytest.mark.parametrize("prec,basis16", [(dd.DD_PREC_FP16, 0), (dd.DD_PREC_FP32, 0), (dd.DD_PREC_FP16, 1)],
                         ids=["mixed", "fp32", "mixed_fp16basis"])
def test_benchmark_solve_true_residual_by_oracle(bench_lattice, prec, basis16):
    """The solve the benchmark times: 32^3x64, width 0.5 + 5 APE steps, kappa 0.136,
    c_sw 1.5, 8x4x4x4 domains, (I_Schwarz, I_domain, m, k) = (2, 4, 40, 8), two threads per
    site, device-resident f and x (the benchmark's call), in the mixed form (FP16 storage
    in the Schwarz kernel), the plain FP32 form and the mixed form with an FP16 Krylov
    basis.  The oracle recomputes |f - A x| / |f| in FP64 on the whole lattice from the
    returned x."""
    w, c, U, F, f = bench_lattice
    fd = torch.view_as_real(torch.from_numpy(f)).cuda().contiguous()
    xd = torch.zeros_like(fd)
    info = c.dd_solve(fd, xd, where=dd.DD_DEVICE, tol=w.tol, m=w.m, k=w.k, max_iter=2000,
                      i_schwarz=w.i_schwarz, i_domain=w.i_domain, storage_prec=prec, basis_fp16=basis16)
    x = torch.view_as_complex(xd.cpu()).numpy()
    r = f - W.apply_A(U, x, w.kappa, w.csw, F)
    res = float(np.linalg.norm(r) / np.linalg.norm(f))
    print(f"32^3x64 kappa {w.kappa}: {info.iterations} it, library {info.true_rel_residual:.3e}, oracle {res:.3e}")
    assert info.true_rel_residual <= 1e-10
    assert res <= 1e-10


def test_solve_after_schwarz_state_grows_matches_fresh_context():
    """Captured Arnoldi-step graphs hold the Schwarz state's addresses.  A batched call with
    more right-hand sides reallocates that state; the graphs must be rebuilt, so a solve
    after it equals, bit for bit, the same solve on a fresh context."""
    dims, dom = (16, 8, 8, 8), (8, 4, 4, 4)
    U = gauge(dims, 0.5, 31, ape=2)
    f = synth.gaussian_source(dims, 32)
    kw = dict(tol=1e-10, m=8, k=2, i_schwarz=2, i_domain=3, storage_prec=dd.DD_PREC_FP16)
    c = ctx_for(dims, dom, U, 0.1250, 1.5)
    x1 = np.zeros_like(f)
    info = c.dd_solve(f, x1, **kw)
    assert info.restarts >= 1          # some Arnoldi steps were replayed from graphs
    nb = c.dd_spinor_bytes(dd.DD_PREC_FP32, dd.DD_LAYOUT_INTERNAL)
    fs = [synth.gaussian_source(dims, 40 + r) for r in range(3)]
    src = torch.empty(3 * nb, dtype=torch.uint8, device="cuda")
    for r, fr in enumerate(fs):
        c.dd_pack_spinor(torch.view_as_real(torch.from_numpy(fr)).cuda().contiguous(), dd.DD_PREC_FP64,
                         src[r * nb:(r + 1) * nb], dd.DD_PREC_FP32)
    out = torch.empty_like(src)
    c.dd_sap_precondition_batch(src, out, 3, 2, 3, dd.DD_PREC_FP16)
    x2 = np.zeros_like(f)
    c.dd_solve(f, x2, **kw)
    fresh = ctx_for(dims, dom, U, 0.1250, 1.5)
    x3 = np.zeros_like(f)
    fresh.dd_solve(f, x3, **kw)
    assert np.array_equal(x2, x3)
    assert np.array_equal(x1, x3)


def test_solve_with_additive_schwarz():
    """FGMRES-DR preconditioned by the additive form reaches the target on the 8^4
    workload; the oracle certifies the residual."""
    w = synth.WORKLOADS["8^4"]
    U = synth.make_gauge(w).numpy()
    f = synth.make_sources(w)[0]
    c = ctx_for(w.dims, w.domain, U, w.kappa, w.csw)
    x = np.zeros_like(f)
    info = c.dd_solve(f, x, tol=w.tol, m=w.m, k=w.k, i_schwarz=w.i_schwarz, i_domain=w.i_domain, additive=1)
    assert S.true_residual(U, x, f, w.kappa, w.csw) <= 1e-10 and info.true_rel_residual <= 1e-10


@pytest.mark.parametrize("additive", [0, 1], ids=["multiplicative", "additive"])
def test_gcr_solve(additive):
    """Flexible GCR around the Schwarz preconditioner (SAP-GCR, Sec. V): the oracle's FP64
    true residual <= 1e-10 and the same solution as FGMRES-DR within the conditioning."""
    w = synth.WORKLOADS["8^4"]
    U = synth.make_gauge(w).numpy()
    f = synth.make_sources(w)[0]
    c = ctx_for(w.dims, w.domain, U, w.kappa, w.csw)
    x = np.zeros_like(f)
    info = c.dd_solve_gcr(f, x, tol=1e-10, m=12, max_iter=500, i_schwarz=w.i_schwarz, i_domain=w.i_domain,
                          additive=additive)
    assert S.true_residual(U, x, f, w.kappa, w.csw) <= 1e-10 and info.true_rel_residual <= 1e-10
    xd = np.zeros_like(f)
    c.dd_solve(f, xd, tol=1e-12, m=w.m, k=w.k, i_schwarz=w.i_schwarz, i_domain=w.i_domain)
    assert rel(x, xd) <= 1e-8
