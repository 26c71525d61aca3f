"""The autotuner (dd_autotune; Sec. IV-B: domain size and I_domain chosen by the overall
time-to-solution, Eq. 6-7 for the load of a domain count) on the device, and the solves
it configures: the 16^3x32 lattice alone, and the batched 24^3x48 workload (12 point and
36 Gaussian sources, kappa 0.124) in lockstep with the tuned shape and parameters."""
import numpy as np
import pytest
import torch

import synth
from oracle import wilson as W
from paper_1412_2629_gb300 import dd

from gpu_helpers import ctx_for

pytestmark = pytest.mark.gpu


def _check_choice(w, dom, prm, tps_fixed=0):
    i_s, i_d, prec, tps = prm
    assert all(b in (2, 4, 8) and L % b == 0 and (L // b) % 2 == 0 for b, L in zip(dom, w.dims))
    assert 64 <= int(np.prod(dom)) <= 512
    assert i_s in (1, 2, 4, 8, 16) and 2 <= i_d <= 6 and prec == dd.DD_PREC_FP16
    assert tps in (1, 2) and (tps_fixed == 0 or tps == tps_fixed)


def test_autotune_16x32_and_tuned_solve():
    w = synth.WORKLOADS["16^3x32"]
    kappa = 0.1240
    Ud = synth.make_gauge(w, device="cuda")
    U = Ud.cpu().numpy()
    c = ctx_for(w.dims, w.domain, Ud, kappa, w.csw)
    dom, prm = c.dd_autotune(dd.DD_PREC_FP16)
    print(f"16^3x32: domains {dom}, (I_S, I_d, prec, tps) = {prm}")
    _check_choice(w, dom, prm)
    i_s, i_d, prec, tps = prm
    # a context of the chosen shape: its M reduces the residual of a Gaussian source
    t = ctx_for(w.dims, dom, Ud, kappa, w.csw)
    del Ud
    f = synth.make_sources(w)[0]
    src = torch.view_as_real(torch.from_numpy(f)).to(torch.float32).cuda().contiguous()
    z = torch.empty_like(src)
    t.dd_sap_precondition(src, z, i_s, i_d, prec, dd.DD_LAYOUT_CANONICAL, threads_per_site=tps)
    z64 = z.double()
    Az = torch.empty_like(z64)
    t.dd_apply_D(z64, Az, dd.DD_PREC_FP64, dd.DD_LAYOUT_CANONICAL)
    fd = src.double()
    assert float((fd - Az).norm() / fd.norm()) < 1.0
    # and the solve with the tuned parameters reaches 1e-10, certified by the oracle
    x = np.zeros_like(f)
    t.dd_solve(f, x, tol=1e-10, m=16, k=6, max_iter=3000, i_schwarz=i_s, i_domain=i_d, storage_prec=prec,
               threads_per_site=tps)
    r = f - W.apply_A(U, x, kappa, w.csw)
    assert np.linalg.norm(r) / np.linalg.norm(f) <= 1e-10


def test_batched_workload_autotuned_lockstep():
    """24^3x48 with all 48 sources (12 point, 36 Gaussian) in one lockstep dd_solve, with
    the shape, I_Schwarz, I_domain chosen by dd_autotune (two threads per site fixed:
    the lockstep kernels need it).  Every source's true residual is recomputed with the
    library's FP64 operator; four of them (two point, two Gaussian) by the oracle."""
    w = synth.WORKLOADS["24^3x48"]
    Ud = synth.make_gauge(w, device="cuda")
    c = ctx_for(w.dims, w.domain, Ud, w.kappa, w.csw)
    dom, prm = c.dd_autotune(dd.DD_PREC_FP16, threads_per_site=2)
    print(f"24^3x48: domains {dom}, (I_S, I_d, prec, tps) = {prm}")
    _check_choice(w, dom, prm, tps_fixed=2)
    i_s, i_d, prec, tps = prm
    t = ctx_for(w.dims, dom, Ud, w.kappa, w.csw)
    del c
    U = Ud.cpu().numpy()
    del Ud
    pts = synth.point_sources(w.dims)
    fs = pts + synth.make_sources(w, 36)
    n = len(fs)
    assert n == 48
    fd = torch.stack([torch.view_as_real(torch.from_numpy(f)) for f in fs]).cuda().contiguous()
    xd = torch.zeros_like(fd)
    info = t.dd_solve(fd, xd, nrhs=n, where=dd.DD_DEVICE, tol=w.tol, m=w.m, k=w.k, max_iter=20000,
                      i_schwarz=i_s, i_domain=i_d, storage_prec=prec, threads_per_site=tps)
    print(f"48 sources: {info.iterations} iterations, worst residual {info.true_rel_residual:.2e}, "
          f"{info.t_total:.2f} s")
    assert info.true_rel_residual <= 1e-10
    for r in range(n):
        Ax = torch.empty_like(xd[r])
        t.dd_apply_D(xd[r].contiguous(), Ax, dd.DD_PREC_FP64, dd.DD_LAYOUT_CANONICAL)
        assert float((fd[r] - Ax).norm() / fd[r].norm()) <= 1e-10
    F = W.field_strength(U)
    for r in (0, 7, 12, 47):
        x = torch.view_as_complex(xd[r].cpu()).numpy()
        res = np.linalg.norm(fs[r] - W.apply_A(U, x, w.kappa, w.csw, F)) / np.linalg.norm(fs[r])
        assert res <= 1e-10
