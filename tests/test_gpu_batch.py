"""Several right-hand sides per launch: dd_apply_D_batch and dd_sap_precondition_batch
against one-at-a-time calls and against the oracle (same bars as the single-field tests)."""
import numpy as np
import pytest
import torch

import synth
from oracle import wilson as W
from paper_1412_2629_gb300 import dd

from gpu_helpers import ctx_for, dev, gauge, host, rel

pytestmark = pytest.mark.gpu

DIMS, DOM = (16, 8, 8, 8), (8, 4, 4, 4)


def _pack(c, fields, prec):
    nb = c.dd_spinor_bytes(prec, dd.DD_LAYOUT_INTERNAL)
    buf = torch.empty(len(fields) * nb, dtype=torch.uint8, device="cuda")
    for r, f in enumerate(fields):
        c.dd_pack_spinor(dev(f), dd.DD_PREC_FP64, buf[r * nb:(r + 1) * nb], prec)
    return buf, nb


def _unpack(c, buf, nb, n, prec):
    out = []
    for r in range(n):
        t = torch.empty(DIMS[3], DIMS[2], DIMS[1], DIMS[0], 4, 3, 2, dtype=torch.float64, device="cuda")
        c.dd_unpack_spinor(buf[r * nb:(r + 1) * nb], prec, t, dd.DD_PREC_FP64)
        out.append(host(t))
    return out


@pytest.mark.parametrize("prec,tol", [(dd.DD_PREC_FP32, 1e-6), (dd.DD_PREC_FP16, 3e-3)], ids=["fp32", "fp16"])
def test_apply_batch(prec, tol):
    U = gauge(DIMS, 0.5, 5)
    c = ctx_for(DIMS, DOM, U, 0.1360, 1.5)
    fs = [synth.gaussian_source(DIMS, 200 + r) for r in range(3)]     # odd count: short last pair
    src, nb = _pack(c, fs, prec)
    out = torch.empty_like(src)
    c.dd_apply_D_batch(src, out, len(fs), prec)
    got = _unpack(c, out, nb, len(fs), prec)
    for r, f in enumerate(fs):
        assert rel(got[r], W.apply_A(U, f, 0.1360, 1.5)) <= tol
        one = torch.empty(nb, dtype=torch.uint8, device="cuda")
        c.dd_apply_D(src[r * nb:(r + 1) * nb], one, prec, dd.DD_LAYOUT_INTERNAL)
        assert rel(got[r], _unpack(c, one, nb, 1, prec)[0]) <= 1e-6


@pytest.mark.parametrize("prec", [dd.DD_PREC_FP32, dd.DD_PREC_FP16], ids=["fp32", "fp16"])
def test_sap_batch_equals_single(prec):
    U = gauge(DIMS, 0.5, 6)
    c = ctx_for(DIMS, DOM, U, 0.1300, 1.5)
    fs = [synth.gaussian_source(DIMS, 300 + r) for r in range(3)]
    src, nb = _pack(c, fs, dd.DD_PREC_FP32)
    out = torch.empty_like(src)
    c.dd_sap_precondition_batch(src, out, len(fs), 3, 4, prec)
    for r in range(len(fs)):
        one = torch.empty(nb, dtype=torch.uint8, device="cuda")
        c.dd_sap_precondition(src[r * nb:(r + 1) * nb], one, 3, 4, prec, dd.DD_LAYOUT_INTERNAL)
        a = out[r * nb:(r + 1) * nb].view(torch.float32).double()
        b = one.view(torch.float32).double()
        assert float((a - b).norm() / b.norm()) <= 1e-6


def test_sap_lattices_in_one_launch_match_oracle():
    """Three lattices of different volume (own gauge field, clover and kappa) with three
    right-hand sides each, in one launch per half-sweep: every output equals the oracle's
    multiplicative SAP on its own lattice (FP16 storage bar, 5e-3) and, to 1e-6, what the
    lattice gives alone."""
    from oracle import dd as DD
    shapes = [((8, 8, 8, 8), 0.1250, 41), ((8, 8, 8, 16), 0.1300, 42), ((16, 8, 8, 8), 0.1350, 43)]
    nr, i_s, i_d = 3, 3, 4
    ctxs, ins, outs, refs, want = [], [], [], [], []
    for dims, kappa, seed in shapes:
        U = gauge(dims, 0.5, seed)
        c = ctx_for(dims, (4, 4, 4, 4), U, kappa, 1.5)
        fs = [synth.gaussian_source(dims, seed + 1 + r) for r in range(nr)]
        src, nb = _pack(c, fs, dd.DD_PREC_FP32)
        ref = torch.empty_like(src)
        c.dd_sap_precondition_batch(src, ref, nr, i_s, i_d, dd.DD_PREC_FP16)
        F = W.field_strength(U)
        dom = DD.Domains(dims, (4, 4, 4, 4))
        want.append([DD.sap(U, F, f, kappa, 1.5, dom, i_s, i_d) for f in fs])
        ctxs.append(c)
        ins.append(src)
        outs.append(torch.empty_like(src))
        refs.append(ref)
    dd.dd_sap_precondition_lattices(ctxs, ins, outs, i_s, i_d, nrhs=nr)
    for c, (dims, _, _), o, r, wl in zip(ctxs, shapes, outs, refs, want):
        nb = c.dd_spinor_bytes(dd.DD_PREC_FP32, dd.DD_LAYOUT_INTERNAL)
        a, b = o.view(torch.float32).double(), r.view(torch.float32).double()
        assert float((a - b).norm() / b.norm()) <= 1e-6
        for k, u in enumerate(wl):
            t = torch.empty(dims[3], dims[2], dims[1], dims[0], 4, 3, 2, dtype=torch.float32, device="cuda")
            c.dd_unpack_spinor(o[k * nb:(k + 1) * nb], dd.DD_PREC_FP32, t, dd.DD_PREC_FP32)
            assert rel(host(t), u) <= 5e-3


@pytest.mark.parametrize("prec", [dd.DD_PREC_FP16, dd.DD_PREC_FP16_H2], ids=["fp16", "half2"])
def test_lockstep_solve_equals_sequential(prec, monkeypatch):
    """dd_solve with several right-hand sides runs them in lockstep (one Schwarz launch per
    half-sweep and one operator launch per Arnoldi step for all of them, each with its
    own basis and restarts).  It must give what one solve after another gives: every true
    residual <= 1e-10 (oracle, FP64), solutions within 1e-8, a zero source left at zero.
    A weak preconditioner (I_S = 1, I_d = 2) with m = 8, k = 3 needs about three cycles,
    so deflated restarts happen at different steps for different sources."""
    from oracle import solve as S
    dims, dom, kappa, csw = (16, 8, 8, 8), (8, 4, 4, 4), 0.1300, 1.0   # the field recipe of the 8^4 workload
    U = gauge(dims, 0.6, 31)
    fs = [synth.gaussian_source(dims, 40 + r) for r in range(4)] + [np.zeros_like(synth.gaussian_source(dims, 1))]
    fs[2] = synth.point_sources(dims)[5]
    f = np.stack(fs)
    c = ctx_for(dims, dom, U, kappa, csw)
    kw = dict(tol=1e-10, m=8, k=3, i_schwarz=1, i_domain=2, storage_prec=prec)   # ~18 steps, 3 cycles
    x_lock = np.zeros_like(f)
    info_l = c.dd_solve(f, x_lock, nrhs=len(fs), **kw)
    monkeypatch.setenv("DD_SEQUENTIAL_RHS", "1")
    x_seq = np.zeros_like(f)
    info_s = c.dd_solve(f, x_seq, nrhs=len(fs), **kw)
    for r in range(4):
        assert S.true_residual(U, x_lock[r], f[r], kappa, csw) <= 1e-10
        assert rel(x_lock[r], x_seq[r]) <= 1e-8
    assert not np.any(x_lock[4])
    assert info_l.true_rel_residual <= 1e-10 and info_l.restarts > 0
    assert abs(info_l.iterations - info_s.iterations) <= 2 * len(fs)


def test_lockstep_solve_over_lattices():
    """Three lattices of different volume, two right-hand sides each (one a point source),
    solved in lockstep by dd_solve_lattices: one Schwarz launch per half-sweep covers every
    lattice's unconverged (domain, right-hand side) work.  Every true residual, recomputed
    by the oracle in FP64, is <= 1e-10, and each solution equals the single-lattice
    dd_solve of the same source to 1e-8."""
    from oracle import solve as S
    shapes = [((8, 8, 8, 8), 0.1250, 41), ((8, 8, 8, 16), 0.1300, 42), ((16, 8, 8, 8), 0.1320, 43)]
    kw = dict(tol=1e-10, m=12, k=4, max_iter=2000, i_schwarz=2, i_domain=4)
    ctxs, fs, xs, Us = [], [], [], []
    for dims, kappa, seed in shapes:
        U = gauge(dims, 0.5, seed, ape=2)
        ctxs.append(ctx_for(dims, (4, 4, 4, 4), U, kappa, 1.5))
        fs.append(np.stack([synth.gaussian_source(dims, seed + 1), synth.point_sources(dims)[3]]))
        xs.append(np.zeros_like(fs[-1]))
        Us.append(U)
    info = dd.dd_solve_lattices(ctxs, fs, xs, nrhs=2, **kw)
    assert info.true_rel_residual <= 1e-10
    for (dims, kappa, _), c, U, f, x in zip(shapes, ctxs, Us, fs, xs):
        for r in range(2):
            assert S.true_residual(U, x[r], f[r], kappa, 1.5) <= 1e-10
            x1 = np.zeros_like(f[r])
            c.dd_solve(f[r], x1, storage_prec=dd.DD_PREC_FP16, **kw)
            assert rel(x[r], x1) <= 1e-8
