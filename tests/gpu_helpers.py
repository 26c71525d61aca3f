"""Shared helpers of the GPU parity tests: build contexts through the C ABI and move
canonical fields between numpy (oracle side) and torch device memory (CUDA side)."""
import numpy as np
import torch

import synth
from paper_1412_2629_gb300 import dd


def ctx_for(dims, domain, U, kappa, csw, anti=True):
    c = dd.Context(dims, domain, t_antiperiodic=anti, stream=torch.cuda.current_stream().cuda_stream)
    if isinstance(U, torch.Tensor):
        Ud = U.to("cuda").contiguous()
        c.dd_load_gauge(torch.view_as_real(Ud), dd.DD_DEVICE)
    else:
        c.dd_load_gauge(np.ascontiguousarray(U), dd.DD_HOST)
    c.dd_build_clover(kappa, csw)
    return c


def dev(psi, dtype=torch.float64):
    """Canonical complex spinor (numpy) -> device real tensor [..., 2]."""
    t = torch.from_numpy(np.ascontiguousarray(psi))
    t = torch.view_as_real(t).to(dtype)
    return t.to("cuda").contiguous()


def host(t):
    """Device real tensor [..., 2] -> numpy complex128."""
    a = t.double().cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def gauge(dims, width, seed, ape=0):
    U = synth.random_su3_field(dims, width, seed)
    if ape:
        U = synth.ape_smear(U, 0.5, ape)
    return U.numpy()


def apply_gpu(c, psi, prec):
    """A psi through dd_apply_D: FP64 / FP32 canonical, FP16 via the internal layout."""
    if prec == dd.DD_PREC_FP16:
        src = dev(psi)
        buf = torch.empty(c.dd_spinor_bytes(dd.DD_PREC_FP16, dd.DD_LAYOUT_INTERNAL), dtype=torch.uint8, device="cuda")
        out = torch.empty_like(buf)
        c.dd_pack_spinor(src, dd.DD_PREC_FP64, buf, dd.DD_PREC_FP16)
        c.dd_apply_D(buf, out, dd.DD_PREC_FP16, dd.DD_LAYOUT_INTERNAL)
        res = torch.empty_like(src)
        c.dd_unpack_spinor(out, dd.DD_PREC_FP16, res, dd.DD_PREC_FP64)
        return host(res)
    dt = torch.float64 if prec == dd.DD_PREC_FP64 else torch.float32
    src = dev(psi, dt)
    out = torch.empty_like(src)
    c.dd_apply_D(src, out, prec, dd.DD_LAYOUT_CANONICAL)
    return host(out)
