"""The allocation-free Schwarz entry point, dd_sap_precondition_noalloc.

Some callers cannot call cudaMalloc when they apply the preconditioner: frameworks that
hand out all device memory from their own pool, and loops that cannot afford cudaMalloc's
device-wide synchronisation.  For them
the library keeps the Schwarz working state in one fixed array of its own device memory.
These tests call that entry point through the C ABI twice in a row and check it against
the allocating entry point, dd_sap_precondition, with the tolerances of the Schwarz
parity tests; and check that a lattice too large for the fixed array is refused with a
clear error.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import synth
from paper_1412_2629_gb300 import dd

from gpu_helpers import ctx_for, dev, gauge

pytestmark = pytest.mark.gpu


def _internal(c, f):
    src = dev(f, torch.float32)
    buf = torch.empty(c.dd_spinor_bytes(dd.DD_PREC_FP32, dd.DD_LAYOUT_INTERNAL), dtype=torch.uint8, device="cuda")
    c.dd_pack_spinor(src, dd.DD_PREC_FP32, buf, dd.DD_PREC_FP32)
    return buf


def _rel(a, b):
    a = a.view(torch.float32).double()
    b = b.view(torch.float32).double()
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("prec,tol", [(dd.DD_PREC_FP32, 1e-5), (dd.DD_PREC_FP16, 5e-3)], ids=["fp32", "fp16"])
def test_noalloc_matches_allocating_entry_point(prec, tol):
    dims, dom = (16, 8, 8, 8), (8, 4, 4, 4)
    U = gauge(dims, 0.5, 5)
    c = ctx_for(dims, dom, U, 0.1360, 1.5)
    f = synth.gaussian_source(dims, 105)
    v = _internal(c, f)
    ref = torch.empty_like(v)
    c.dd_sap_precondition(v, ref, 3, 4, prec, dd.DD_LAYOUT_INTERNAL)
    for _ in range(2):
        out = torch.full_like(v, 0xFF)
        c.dd_sap_precondition_noalloc(v, out, 3, 4, prec)
        assert _rel(out, ref) <= tol


def test_noalloc_rejects_lattice_beyond_fixed_array():
    c = dd.Context((32, 32, 32, 64), (8, 4, 4, 4), True, torch.cuda.current_stream().cuda_stream)
    v = torch.zeros(16, dtype=torch.uint8, device="cuda")
    s = c.dd_sap_precondition_noalloc(v, v, 2, 4, dd.DD_PREC_FP16, check=False)
    assert s == dd.DD_ERR_INVALID
    msg = dd.lib().dd_last_error(c._h).decode()
    assert "too large" in msg and "bytes" in msg
