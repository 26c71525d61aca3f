"""GPU parity of the full Wilson-clover operator (Eq. 1-3) against the FP64 oracle.

Bars: FP64 <= 1e-13, FP32 <= 1e-6, FP16 storage <= 3e-3 relative L2 error."""
import numpy as np
import pytest
import torch

import synth
from oracle import wilson as W
from paper_1412_2629_gb300 import dd

from gpu_helpers import apply_gpu, ctx_for, dev, gauge, host, rel

pytestmark = pytest.mark.gpu

CASES = [
    # dims,          domain,        width, seed, kappa, csw, antiperiodic
    ((8, 8, 8, 8), (4, 4, 4, 4), 0.6, 11, 0.1300, 1.0, True),    # the 8^4 workload
    ((16, 8, 8, 8), (8, 4, 4, 4), 0.5, 5, 0.1360, 1.5, True),    # 8x4^3 domains
    ((8, 8, 8, 24), (4, 4, 4, 4), 0.6, 6, 0.1250, 1.7, False),   # 6 domains in t, periodic
    ((8, 16, 8, 8), (4, 8, 2, 4), 0.6, 7, 0.1200, 0.0, True),    # mixed extents, no clover
]
TOL = {dd.DD_PREC_FP64: 1e-13, dd.DD_PREC_FP32: 1e-6, dd.DD_PREC_FP16: 3e-3}


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + "_b" + "x".join(map(str, c[1])))
@pytest.mark.parametrize("prec", [dd.DD_PREC_FP64, dd.DD_PREC_FP32, dd.DD_PREC_FP16], ids=["fp64", "fp32", "fp16"])
def test_apply_matches_oracle(case, prec):
    dims, dom, width, seed, kappa, csw, anti = case
    U = gauge(dims, width, seed)
    psi = synth.gaussian_source(dims, seed + 100)
    want = W.apply_A(U, psi, kappa, csw, bc_t=-1.0 if anti else 1.0)
    c = ctx_for(dims, dom, U, kappa, csw, anti)
    got = apply_gpu(c, psi, prec)
    assert rel(got, want) <= TOL[prec]


def test_pack_unpack_roundtrip_and_point_source():
    dims, dom = (8, 8, 8, 8), (4, 4, 4, 4)
    U = gauge(dims, 0.6, 3)
    c = ctx_for(dims, dom, U, 0.13, 1.0)
    psi = synth.gaussian_source(dims, 4)
    src = dev(psi)
    buf = torch.empty(c.dd_spinor_bytes(dd.DD_PREC_FP64, dd.DD_LAYOUT_INTERNAL), dtype=torch.uint8, device="cuda")
    c.dd_pack_spinor(src, dd.DD_PREC_FP64, buf, dd.DD_PREC_FP64)
    back = torch.empty_like(src)
    c.dd_unpack_spinor(buf, dd.DD_PREC_FP64, back, dd.DD_PREC_FP64)
    assert torch.equal(back, src)
    # point sources at the corner and at the far time boundary touch every wrap
    for site in [(0, 0, 0, 0), (7, 7, 7, 7), (3, 0, 5, 7)]:
        p = np.zeros_like(psi)
        p[site[3], site[2], site[1], site[0], 2, 1] = 1.0
        want = W.apply_A(U, p, 0.13, 1.0)
        assert rel(apply_gpu(c, p, dd.DD_PREC_FP64), want) <= 1e-13


def test_full_size_sampled_sites_32x64():
    """The 32^3x64 workload in the launch configuration the benchmark times (FP32
    and FP16 storage), checked on sampled sites computed one by one by the oracle."""
    w = synth.WORKLOADS["32^3x64"]
    Ud = synth.make_gauge(w, device="cuda")
    c = ctx_for(w.dims, w.domain, Ud, w.kappa, w.csw)
    psi = synth.gaussian_source(w.dims, w.source_seed)
    U = Ud.cpu().numpy()
    del Ud
    rng = np.random.default_rng(0)
    L = w.dims
    coords = [(0, 0, 0, 0), (L[0] - 1, L[1] - 1, L[2] - 1, L[3] - 1), (7, 3, 4, 63), (8, 4, 4, 0)]
    coords += [tuple(int(rng.integers(0, n)) for n in L) for _ in range(28)]
    want = W.apply_A_at(U, psi, w.kappa, w.csw, coords)
    for prec, tol in ((dd.DD_PREC_FP32, 2e-6), (dd.DD_PREC_FP16, 3e-3)):
        got = apply_gpu(c, psi, prec)
        g = np.array([got[t, z, y, x] for (x, y, z, t) in coords])
        assert rel(g, want) <= tol
