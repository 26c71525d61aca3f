"""The non-domain-decomposed comparison solvers (Sec. IV-C, Table III: BiCGstab in double
precision, and a mixed-precision Richardson iteration around BiCGstab), through the
C ABI: solutions certified by the oracle's FP64 true residual, and the same solution as
the domain-decomposed solver within the conditioning of the problem."""
import numpy as np
import pytest

import synth
from oracle import solve as S
from paper_1412_2629_gb300 import dd

from gpu_helpers import ctx_for, gauge, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [dd.DD_PREC_FP64, dd.DD_PREC_FP32], ids=["fp64", "mixed"])
def test_bicgstab_8x4_workload(precision):
    w = synth.WORKLOADS["8^4"]
    U = synth.make_gauge(w).numpy()
    f = synth.make_sources(w)[0]
    c = ctx_for(w.dims, w.domain, U, w.kappa, w.csw)
    x = np.zeros_like(f)
    info = c.dd_solve_bicgstab(f, x, tol=1e-10, max_iter=5000, precision=precision, inner_tol=1e-5)
    res = S.true_residual(U, x, f, w.kappa, w.csw)
    print(f"BiCGstab {precision}: {info.iterations} it, {info.restarts + 1} corrections, residual {res:.2e}")
    assert res <= 1e-10 and info.true_rel_residual <= 1e-10
    if precision == dd.DD_PREC_FP32:
        assert info.restarts >= 1        # several FP64 corrections around FP32 inner solves
    xd = np.zeros_like(f)
    c.dd_solve(f, xd, tol=1e-12, m=w.m, k=w.k, i_schwarz=w.i_schwarz, i_domain=w.i_domain)
    assert rel(x, xd) <= 1e-8


def test_bicgstab_iteration_limit_and_guess():
    dims, dom = (16, 8, 8, 8), (8, 4, 4, 4)
    U = gauge(dims, 0.5, 51, ape=2)
    f = synth.gaussian_source(dims, 52)
    c = ctx_for(dims, dom, U, 0.1240, 1.5)
    x = np.zeros_like(f)
    info = c.dd_solve_bicgstab(f, x, tol=1e-14, max_iter=3, precision=dd.DD_PREC_FP64, check=False)
    assert info.status == dd.DD_ERR_NOT_CONVERGED and info.iterations == 3
    assert 0 < info.true_rel_residual < 1
    # a converged solution as the initial guess: no iterations
    c.dd_solve_bicgstab(f, x, tol=1e-10, max_iter=5000, precision=dd.DD_PREC_FP32)
    info = c.dd_solve_bicgstab(f, x, tol=1e-10, max_iter=5000, precision=dd.DD_PREC_FP64)
    assert info.iterations == 0 and S.true_residual(U, x, f, 0.1240, 1.5) <= 1e-10
