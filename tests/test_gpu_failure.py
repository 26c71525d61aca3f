"""Failure detection through the C ABI, with no GPU fault: shapes the library refuses,
calls in the wrong order, an iteration limit, a non-finite source, and a bounded device
wait that is made to run out (the Schwarz kernel is told to expect 16 bytes that nobody
sends, on a barrier of their own; it gives up after 50 ms, sets an error word, waits for
its real staged copies and returns)."""
import numpy as np
import pytest
import torch

import synth
from paper_1412_2629_gb300 import dd

from gpu_helpers import ctx_for, dev, gauge

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,dom", [
    ((8, 8, 8, 8), (8, 4, 4, 4)),     # L / b = 1
    ((12, 8, 8, 8), (4, 4, 4, 4)),    # L / b = 3, odd
    ((8, 8, 8, 8), (4, 4, 4, 3)),     # extent not a power of two
    ((8, 8, 8, 8), (2, 2, 2, 2)),     # domain of 16 sites: too small for the kernel
])
def test_rejected_shapes(dims, dom):
    with pytest.raises(dd.DDError) as e:
        dd.Context(dims, dom)
    assert e.value.status == dd.DD_ERR_DIMS


def test_wrong_order_and_bad_parameters():
    c = dd.Context((8, 8, 8, 8), (4, 4, 4, 4))
    with pytest.raises(dd.DDError) as e:
        c.dd_build_clover(0.13, 1.0)
    assert e.value.status == dd.DD_ERR_NO_GAUGE
    src = torch.zeros(8 ** 4 * 24, dtype=torch.float32, device="cuda")
    with pytest.raises(dd.DDError) as e:
        c.dd_apply_D(src, src.clone(), dd.DD_PREC_FP32)
    assert e.value.status == dd.DD_ERR_NO_CLOVER
    U = gauge((8, 8, 8, 8), 0.6, 3)
    c.dd_load_gauge(U, dd.DD_HOST)
    c.dd_build_clover(0.13, 1.0)
    with pytest.raises(dd.DDError) as e:
        c.dd_sap_precondition(src, src.clone(), 0, 4, dd.DD_PREC_FP16)
    assert e.value.status == dd.DD_ERR_INVALID


def test_iteration_limit_and_nonfinite_source():
    w = synth.WORKLOADS["8^4"]
    U = synth.make_gauge(w).numpy()
    c = ctx_for(w.dims, w.domain, U, w.kappa, w.csw)
    f = synth.make_sources(w)[0]
    x = np.zeros_like(f)
    info = c.dd_solve(f, x, tol=1e-14, m=4, k=0, max_iter=1, i_schwarz=1, i_domain=1, check=False)
    assert info.status == dd.DD_ERR_NOT_CONVERGED and info.iterations == 1
    assert 0 < info.true_rel_residual < 1
    bad = f.copy()
    bad[0, 0, 0, 0, 0, 0] = np.nan
    info = c.dd_solve(bad, np.zeros_like(f), check=False)
    assert info.status == dd.DD_ERR_NONFINITE


def test_bounded_wait_runs_out_and_context_stays_usable(monkeypatch):
    dims, dom = (16, 8, 8, 8), (8, 4, 4, 4)
    U = gauge(dims, 0.5, 5)
    f = synth.gaussian_source(dims, 7)
    monkeypatch.setenv("DD_INJECT_WAIT_TIMEOUT", "1")
    c = ctx_for(dims, dom, U, 0.13, 1.0)
    monkeypatch.delenv("DD_INJECT_WAIT_TIMEOUT")
    src = dev(f, torch.float32)
    with pytest.raises(dd.DDError) as e:
        c.dd_sap_precondition(src, torch.empty_like(src), 1, 2, dd.DD_PREC_FP16)
    assert e.value.status == dd.DD_ERR_TIMEOUT
    # the allocation-free entry point runs the same kernel on its fixed array: same status
    nb = c.dd_spinor_bytes(dd.DD_PREC_FP32, dd.DD_LAYOUT_INTERNAL)
    vi = torch.empty(nb, dtype=torch.uint8, device="cuda")
    c.dd_pack_spinor(src, dd.DD_PREC_FP32, vi, dd.DD_PREC_FP32)
    s = c.dd_sap_precondition_noalloc(vi, torch.empty_like(vi), 1, 2, dd.DD_PREC_FP16, check=False)
    assert s == dd.DD_ERR_TIMEOUT
    # a fresh context on the same GPU works, and so does the operator of the first one
    ok = ctx_for(dims, dom, U, 0.13, 1.0)
    out = torch.empty_like(src)
    ok.dd_sap_precondition(src, out, 1, 2, dd.DD_PREC_FP16)
    assert torch.isfinite(out).all()
    c.dd_apply_D(src, torch.empty_like(src), dd.DD_PREC_FP32)
