"""The other workload shapes: 24^3x48 with point and Gaussian sources (batched right-hand
sides) and a 16^3x32 lattice, true residuals recomputed by the oracle in FP64; the
near-critical 48^3x96 lattice at full size, with the FP64 operator that certifies its
residual checked against the oracle site by site on the solution itself."""
import numpy as np
import pytest
import torch

import synth
from oracle import solve as S
from oracle import wilson as W
from paper_1412_2629_gb300 import dd

from gpu_helpers import ctx_for

pytestmark = pytest.mark.gpu


def test_24x48_point_and_gaussian_sources():
    w = synth.WORKLOADS["24^3x48"]
    Ud = synth.make_gauge(w, device="cuda")
    U = Ud.cpu().numpy()
    c = ctx_for(w.dims, w.domain, Ud, w.kappa, w.csw)
    del Ud
    pts = synth.point_sources(w.dims)
    fs = [pts[0], pts[7]] + synth.make_sources(w, 2)   # two of the 12 point sources, two Gaussian
    f = np.stack(fs)
    x = np.zeros_like(f)
    info = c.dd_solve(f, x, nrhs=len(fs), tol=w.tol, m=w.m, k=w.k, i_schwarz=w.i_schwarz, i_domain=w.i_domain)
    assert info.true_rel_residual <= 1e-10
    for r in range(len(fs)):
        assert S.true_residual(U, x[r], f[r], w.kappa, w.csw) <= 1e-10


def test_16x32_lattice_solve():
    w = synth.WORKLOADS["16^3x32"]
    Ud = synth.make_gauge(w, device="cuda")
    U = Ud.cpu().numpy()
    c = ctx_for(w.dims, w.domain, Ud, 0.1240, w.csw)
    del Ud
    f = synth.make_sources(w)[0]
    x = np.zeros_like(f)
    c.dd_solve(f, x, tol=1e-10, m=16, k=6, i_schwarz=16, i_domain=5)
    assert S.true_residual(U, x, f, 0.1240, w.csw) <= 1e-10


def test_48x96_near_critical_solve():
    """FGMRES-DR(32, 8) with the mixed Schwarz preconditioner at kappa just below the
    field's critical value: |f - A x| / |f| <= 1e-10 with the library's FP64 operator,
    and that operator applied to the solution equals the oracle's A x on 64 sampled
    sites (one by one, FP64) to 1e-12."""
    w = synth.WORKLOADS["48^3x96"]
    Ud = synth.make_gauge(w, device="cuda")
    c = ctx_for(w.dims, w.domain, Ud, w.kappa, w.csw)
    U = Ud.cpu().numpy()
    del Ud
    f = synth.make_sources(w)[0]
    fd = torch.view_as_real(torch.from_numpy(f)).cuda().contiguous()
    xd = torch.zeros_like(fd)
    info = c.dd_solve(fd, xd, where=dd.DD_DEVICE, tol=w.tol, m=w.m, k=w.k, max_iter=20000,
                      i_schwarz=w.i_schwarz, i_domain=w.i_domain)
    Ax = torch.empty_like(xd)
    c.dd_apply_D(xd, Ax, dd.DD_PREC_FP64, dd.DD_LAYOUT_CANONICAL)
    r = float((fd - Ax).norm() / fd.norm())
    assert r <= 1e-10 and info.true_rel_residual <= 1e-10
    x = torch.view_as_complex(xd.cpu()).numpy()
    Axh = torch.view_as_complex(Ax.cpu()).numpy()
    rng = np.random.default_rng(5)
    coords = [tuple(int(rng.integers(0, L)) for L in w.dims) for _ in range(64)]
    coords += [(0, 0, 0, 0), (47, 47, 47, 95), (0, 0, 0, 95)]   # wraps in every direction, time boundary
    want = W.apply_A_at(U, x, w.kappa, w.csw, coords)
    got = np.stack([Axh[t, z, y, xx] for (xx, y, z, t) in coords])
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
