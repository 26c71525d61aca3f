"""GPU parity of the Schwarz preconditioner M (Sec. II-D, Table I) against the oracle's
multiplicative SAP with the same domains, colours and MR step count.

Bars (MR step lengths depend on the data, so rounding compounds mildly): FP32 storage
<= 1e-5, FP16 storage <= 5e-3 relative L2.  FP16 storage with packed FP16 products
(DD_PREC_FP16_H2) is held to the same 5e-3: its products round to FP16 (u = 2^-11) like
the FP16-stored operands they multiply, and the error measured against the oracle is
0.9-1.0e-3 on these cases.

The cases span one partial wave of CTAs (8 to 96 domains per colour) up to several waves
(32x32x16x16 with 8x4x4x4 domains: 256 domains per colour on 152 SMs, one CTA per SM, as
in the benchmark's launches)."""
import numpy as np
import pytest
import torch

import synth
from oracle import dd as DD
from oracle import wilson as W
from paper_1412_2629_gb300 import dd

from gpu_helpers import ctx_for, dev, gauge, host, rel

pytestmark = pytest.mark.gpu


def sap_gpu(c, f, i_s, i_d, prec, tps=0):
    src = dev(f, torch.float32)
    out = torch.empty_like(src)
    c.dd_sap_precondition(src, out, i_s, i_d, prec, dd.DD_LAYOUT_CANONICAL, threads_per_site=tps)
    return host(out)


CASES = [
    ((8, 8, 8, 8), (4, 4, 4, 4), 0.6, 11, 0.1300, 1.0, True, 16, 4),
    ((16, 8, 8, 8), (8, 4, 4, 4), 0.5, 5, 0.1360, 1.5, True, 3, 5),
    ((8, 8, 8, 24), (4, 4, 4, 4), 0.6, 6, 0.1250, 1.7, False, 2, 3),
    ((8, 16, 8, 8), (4, 8, 2, 4), 0.6, 7, 0.1200, 1.1, True, 2, 2),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + "_b" + "x".join(map(str, c[1])))
def test_sap_matches_oracle(case):
    dims, dom, width, seed, kappa, csw, anti, i_s, i_d = case
    U = gauge(dims, width, seed)
    f = synth.gaussian_source(dims, seed + 7)
    F = W.field_strength(U)
    bc = -1.0 if anti else 1.0
    doms = DD.Domains(dims, dom)
    solver = DD.BlockSolver(U, F, kappa, csw, doms)
    # the oracle's SAP with the chosen boundary condition
    u = np.zeros_like(f)
    for _ in range(i_s):
        for colour in (0, 1):
            r = f - W.apply_A(U, u, kappa, csw, F, bc_t=bc)
            u = u + solver_solve(solver, r, colour, i_d, U, bc)
    c = ctx_for(dims, dom, U, kappa, csw, anti)
    for tps in (1, 2):   # one thread per site, or hop directions and chirality split over two
        got32 = sap_gpu(c, f, i_s, i_d, dd.DD_PREC_FP32, tps)
        assert rel(got32, u) <= 1e-5
        got16 = sap_gpu(c, f, i_s, i_d, dd.DD_PREC_FP16, tps)
        assert rel(got16, u) <= 5e-3
    goth2 = sap_gpu(c, f, i_s, i_d, dd.DD_PREC_FP16_H2, 2)
    print(f"half2 products: rel L2 {rel(goth2, u):.2e} against the oracle")
    assert rel(goth2, u) <= 5e-3


def solver_solve(solver, r, colour, i_d, U, bc):
    if bc == -1.0:
        return solver.solve(r, colour, i_d)
    # periodic time boundary: same block solver with the hops evaluated periodically
    orig = solver.hop_in
    solver.hop_in = lambda v: -0.5 * W.hopping(U, v, bc_t=bc, keep=solver.dom.keep_inside)
    try:
        return solver.solve(r, colour, i_d)
    finally:
        solver.hop_in = orig


def test_sap_full_size_properties():
    """On the 32^3x64 workload, in the launch configuration of the benchmark: with the
    Schwarz parameters the solver uses there (I_Schwarz = 2, I_domain = 4) M reduces the
    residual, |f - A M f| < |f|, and the FP16-storage result stays within 5e-3 of the
    FP32 one (also with packed FP16 products).  With the paper's I_Schwarz = 16 the multiplicative iteration is not a
    contraction on this workload (kappa = 0.136 lies above the critical kappa of these
    smooth synthetic fields), which the oracle shows on an 8^4 lattice of the same kind."""
    w = synth.WORKLOADS["32^3x64"]
    Ud = synth.make_gauge(w, device="cuda")
    c = ctx_for(w.dims, w.domain, Ud, w.kappa, w.csw)
    del Ud
    f = synth.gaussian_source(w.dims, w.source_seed)
    z = {}
    for prec in (dd.DD_PREC_FP32, dd.DD_PREC_FP16, dd.DD_PREC_FP16_H2):
        src = dev(f, torch.float32)
        out = torch.empty_like(src)
        c.dd_sap_precondition(src, out, 2, 4, prec, dd.DD_LAYOUT_CANONICAL)
        z64 = out.double()
        Az = torch.empty_like(z64)
        c.dd_apply_D(z64, Az, dd.DD_PREC_FP64, dd.DD_LAYOUT_CANONICAL)
        r = (dev(f) - Az).norm() / dev(f).norm()
        assert float(r) < 0.9
        z[prec] = z64
    d = (z[dd.DD_PREC_FP16] - z[dd.DD_PREC_FP32]).norm() / z[dd.DD_PREC_FP32].norm()
    assert float(d) <= 5e-3
    d2 = (z[dd.DD_PREC_FP16_H2] - z[dd.DD_PREC_FP32]).norm() / z[dd.DD_PREC_FP32].norm()
    print(f"32^3x64: FP16 storage {float(d):.2e}, half2 products {float(d2):.2e} from FP32")
    assert float(d2) <= 5e-3


def test_sap_several_waves_matches_oracle():
    """32x32x16x16 lattice of the 32^3x64 workload's kind (width 0.5 + 5 APE steps, kappa
    0.136, c_sw 1.5) with its 8x4x4x4 domains: 512 domains, 256 per colour, so each
    half-sweep runs 1.7 waves of one CTA per SM on 152 SMs.  I_Schwarz = 2 and I_domain = 4
    as in the benchmark, so the second sweep reads the stored residual and the faces.  All
    storage forms and both thread layouts against one oracle application."""
    dims, dom = (32, 32, 16, 16), (8, 4, 4, 4)
    kappa, csw, i_s, i_d = 0.1360, 1.5, 2, 4
    Ud = synth.random_su3_field(dims, 0.5, 61, device="cuda")
    Ud = synth.ape_smear(Ud, 0.5, 5)
    U = Ud.cpu().numpy()
    f = synth.gaussian_source(dims, 62)
    c = ctx_for(dims, dom, Ud, kappa, csw)
    del Ud
    got = {}
    for prec, tps in ((dd.DD_PREC_FP32, 1), (dd.DD_PREC_FP32, 2), (dd.DD_PREC_FP16, 1), (dd.DD_PREC_FP16, 2),
                      (dd.DD_PREC_FP16_H2, 2)):
        got[(prec, tps)] = sap_gpu(c, f, i_s, i_d, prec, tps)
    F = W.field_strength(U)
    u = DD.sap(U, F, f, kappa, csw, DD.Domains(dims, dom), i_s, i_d)
    bars = {dd.DD_PREC_FP32: 1e-5, dd.DD_PREC_FP16: 5e-3, dd.DD_PREC_FP16_H2: 5e-3}
    for (prec, tps), z in got.items():
        e = rel(z, u)
        print(f"storage {prec} tps {tps}: rel L2 {e:.2e}")
        assert e <= bars[prec]


@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: "x".join(map(str, c[0])) + "_b" + "x".join(map(str, c[1])))
def test_additive_sap_matches_oracle(case):
    """The additive form (block Jacobi, Sec. II-D Eq. 4): one launch per sweep over both
    colours, faces double-buffered; against the oracle's additive SAP with the same
    domains and MR steps, at the multiplicative form's bars."""
    dims, dom, width, seed, kappa, csw, anti, i_s, i_d = case
    if not anti:
        pytest.skip("the oracle's additive SAP uses the antiperiodic time boundary")
    U = gauge(dims, width, seed)
    f = synth.gaussian_source(dims, seed + 7)
    F = W.field_strength(U)
    u = DD.sap_additive(U, F, f, kappa, csw, DD.Domains(dims, dom), i_s, i_d)
    c = ctx_for(dims, dom, U, kappa, csw, anti)
    for prec, bar in ((dd.DD_PREC_FP32, 1e-5), (dd.DD_PREC_FP16, 5e-3), (dd.DD_PREC_FP16_H2, 5e-3)):
        src = dev(f, torch.float32)
        out = torch.empty_like(src)
        c.dd_sap_precondition(src, out, i_s, i_d, prec, dd.DD_LAYOUT_CANONICAL, additive=1)
        e = rel(host(out), u)
        print(f"additive storage {prec}: rel L2 {e:.2e}")
        assert e <= bar
