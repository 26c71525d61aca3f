"""The other workload shapes: 24^3x48 with point and Gaussian sources (batched right-hand
sides) and a 16^3x32 lattice; true residuals recomputed by the oracle in FP64."""
import numpy as np
import pytest

import synth
from oracle import solve as S
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
