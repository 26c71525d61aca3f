"""ctypes binding of include/dd.h: argument marshalling only.

Every numerical step runs in libdd.so.  Loading fails loudly if the library has not
been built (python -m paper_1412_2629_gb300.build); there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdd.so")

DD_OK = 0
DD_ERR_INVALID, DD_ERR_DIMS, DD_ERR_NO_GAUGE, DD_ERR_NO_CLOVER = 1, 2, 3, 4
DD_ERR_SINGULAR_CLOVER, DD_ERR_NOT_CONVERGED, DD_ERR_NONFINITE = 5, 6, 7
DD_ERR_TIMEOUT, DD_ERR_OOM, DD_ERR_CUDA = 8, 9, 10
DD_PREC_FP64, DD_PREC_FP32, DD_PREC_FP16, DD_PREC_FP16_H2 = 0, 1, 2, 3
DD_HOST, DD_DEVICE = 0, 1
DD_LAYOUT_CANONICAL, DD_LAYOUT_INTERNAL = 0, 1


class dd_sap_params(C.Structure):
    _fields_ = [("i_schwarz", C.c_int), ("i_domain", C.c_int), ("storage_prec", C.c_int),
                ("threads_per_site", C.c_int), ("additive", C.c_int)]


class dd_solve_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("m", C.c_int), ("k", C.c_int), ("max_iter", C.c_int),
                ("sap", dd_sap_params), ("basis_fp16", C.c_int)]


class dd_bicgstab_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("precision", C.c_int), ("inner_tol", C.c_double)]


class dd_mg_params(C.Structure):
    _fields_ = [("n_tv", C.c_int), ("setup_iters", C.c_int), ("coarse_m", C.c_int), ("coarse_cycles", C.c_int),
                ("smoother", dd_sap_params), ("setup_mode", C.c_int)]


class dd_solve_info(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("restarts", C.c_int),
                ("reliable_updates", C.c_int), ("deflated_restarts", C.c_int),
                ("true_rel_residual", C.c_double), ("t_total", C.c_double), ("t_A", C.c_double),
                ("t_M", C.c_double), ("t_GS", C.c_double), ("t_other", C.c_double),
                ("flops_nominal", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class DDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"dd status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1412_2629_gb300.build`")
        L = C.CDLL(LIB_PATH)
        P, I, D = C.c_void_p, C.c_int, C.c_double
        sig = {
            "dd_create": (I, [C.POINTER(P), C.POINTER(I), C.POINTER(I), I, P]),
            "dd_destroy": (I, [P]),
            "dd_last_error": (C.c_char_p, [P]),
            "dd_load_gauge": (I, [P, P, I]),
            "dd_build_clover": (I, [P, D, D]),
            "dd_apply_D": (I, [P, P, P, I, I]),
            "dd_sap_precondition": (I, [P, P, P, C.POINTER(dd_sap_params), I]),
            "dd_sap_precondition_noalloc": (I, [P, P, P, C.POINTER(dd_sap_params)]),
            "dd_sap_precondition_batch": (I, [P, P, P, I, C.POINTER(dd_sap_params)]),
            "dd_apply_D_batch": (I, [P, P, P, I, I]),
            "dd_sap_precondition_lattices": (I, [C.POINTER(P), C.POINTER(P), C.POINTER(P), I, I,
                                                 C.POINTER(dd_sap_params)]),
            "dd_solve": (I, [P, P, P, I, I, C.POINTER(dd_solve_params), C.POINTER(dd_solve_info)]),
            "dd_solve_bicgstab": (I, [P, P, P, I, C.POINTER(dd_bicgstab_params), C.POINTER(dd_solve_info)]),
            "dd_solve_gcr": (I, [P, P, P, I, C.POINTER(dd_solve_params), C.POINTER(dd_solve_info)]),
            "dd_solve_lattices": (I, [C.POINTER(P), I, C.POINTER(P), C.POINTER(P), I, I,
                                      C.POINTER(dd_solve_params), C.POINTER(dd_solve_info)]),
            "dd_spinor_bytes": (C.c_size_t, [P, I, I]),
            "dd_pack_spinor": (I, [P, P, I, P, I]),
            "dd_unpack_spinor": (I, [P, P, I, P, I]),
            "dd_launch_count": (C.c_longlong, [P]),
            "dd_load_model": (D, [C.c_longlong, I]),
            "dd_autotune": (I, [P, I, C.POINTER(I), C.POINTER(dd_sap_params)]),
            "dd_deflate_host": (I, [I, I, P, P, P, P, P, P, P]),
            "dd_deflate_device": (I, [I, I, P, P, P, P, P, P, P, C.POINTER(D)]),
            "dd_fp32_peak": (I, [I, C.POINTER(D), C.POINTER(D)]),
            "dd_fp64_peak": (I, [I, C.POINTER(D), C.POINTER(D)]),
            "dd_mg_setup": (I, [P, P, I, C.POINTER(dd_mg_params), C.POINTER(D)]),
            "dd_mg_restrict": (I, [P, P, P]),
            "dd_mg_prolong": (I, [P, P, P]),
            "dd_mg_coarse_apply": (I, [P, P, P]),
            "dd_mg_coarse_solve": (I, [P, P, P]),
            "dd_mg_precondition": (I, [P, P, P, I]),
            "dd_solve_mg": (I, [P, P, P, I, C.POINTER(dd_solve_params), C.POINTER(dd_solve_info)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _ptr(x):
    """Address of a numpy array or torch tensor (host or device)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x)


def _ints(v):
    return (C.c_int * 4)(*[int(a) for a in v])


class Context:
    """Owner of one dd_ctx.  All calls map one to one onto the C ABI."""

    def __init__(self, dims, domain, t_antiperiodic=True, stream=None):
        self._h = C.c_void_p()
        s = lib().dd_create(C.byref(self._h), _ints(dims), _ints(domain), int(bool(t_antiperiodic)),
                            C.c_void_p(stream) if stream else None)
        if s != DD_OK:
            raise DDError(s, "dd_create rejected the lattice / domain shape")
        self.dims, self.domain = tuple(dims), tuple(domain)

    def close(self):
        if self._h:
            lib().dd_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s):
        if s != DD_OK:
            raise DDError(s, lib().dd_last_error(self._h).decode())
        return s

    def dd_load_gauge(self, U, where=DD_HOST):
        return self._check(lib().dd_load_gauge(self._h, _ptr(U), where))

    def dd_build_clover(self, kappa, csw):
        return self._check(lib().dd_build_clover(self._h, float(kappa), float(csw)))

    def dd_apply_D(self, inp, out, prec, layout=DD_LAYOUT_CANONICAL):
        return self._check(lib().dd_apply_D(self._h, _ptr(inp), _ptr(out), prec, layout))

    def dd_sap_precondition(self, inp, out, i_schwarz, i_domain, storage_prec, layout=DD_LAYOUT_CANONICAL,
                            threads_per_site=0, additive=0):
        p = dd_sap_params(i_schwarz, i_domain, storage_prec, threads_per_site, additive)
        return self._check(lib().dd_sap_precondition(self._h, _ptr(inp), _ptr(out), C.byref(p), layout))

    def dd_sap_precondition_batch(self, inp, out, nrhs, i_schwarz, i_domain, storage_prec, threads_per_site=0,
                                  additive=0):
        """nrhs internal-layout FP32 fields one after another; one launch per half-sweep."""
        p = dd_sap_params(i_schwarz, i_domain, storage_prec, threads_per_site, additive)
        return self._check(lib().dd_sap_precondition_batch(self._h, _ptr(inp), _ptr(out), nrhs, C.byref(p)))

    def dd_apply_D_batch(self, inp, out, nrhs, prec):
        """nrhs internal-layout fields (FP32 or FP16) one after another."""
        return self._check(lib().dd_apply_D_batch(self._h, _ptr(inp), _ptr(out), nrhs, prec))

    def dd_sap_precondition_noalloc(self, inp, out, i_schwarz, i_domain, storage_prec, check=True,
                                    threads_per_site=0):
        """Internal-layout FP32 in/out; no device allocation (fixed scratch array)."""
        p = dd_sap_params(i_schwarz, i_domain, storage_prec, threads_per_site)
        s = lib().dd_sap_precondition_noalloc(self._h, _ptr(inp), _ptr(out), C.byref(p))
        return self._check(s) if check else s

    def dd_solve(self, f, x, nrhs=1, where=DD_HOST, tol=1e-10, m=16, k=0, max_iter=1000, i_schwarz=16,
                 i_domain=4, storage_prec=DD_PREC_FP16, check=True, threads_per_site=0, additive=0, basis_fp16=0):
        p = dd_solve_params(tol, m, k, max_iter,
                            dd_sap_params(i_schwarz, i_domain, storage_prec, threads_per_site, additive), basis_fp16)
        info = dd_solve_info()
        s = lib().dd_solve(self._h, _ptr(f), _ptr(x), nrhs, where, C.byref(p), C.byref(info))
        if check:
            self._check(s)
        return info

    def dd_solve_gcr(self, f, x, where=DD_HOST, tol=1e-10, m=16, max_iter=1000, i_schwarz=16, i_domain=4,
                     storage_prec=DD_PREC_FP16, check=True, threads_per_site=0, additive=0):
        p = dd_solve_params(tol, m, 0, max_iter,
                            dd_sap_params(i_schwarz, i_domain, storage_prec, threads_per_site, additive))
        info = dd_solve_info()
        s = lib().dd_solve_gcr(self._h, _ptr(f), _ptr(x), where, C.byref(p), C.byref(info))
        if check:
            self._check(s)
        return info

    def dd_solve_bicgstab(self, f, x, where=DD_HOST, tol=1e-10, max_iter=10000, precision=DD_PREC_FP64,
                          inner_tol=1e-5, check=True):
        p = dd_bicgstab_params(tol, max_iter, precision, inner_tol)
        info = dd_solve_info()
        s = lib().dd_solve_bicgstab(self._h, _ptr(f), _ptr(x), where, C.byref(p), C.byref(info))
        if check:
            self._check(s)
        return info

    def dd_mg_setup(self, tv, n_tv, where=DD_HOST, setup_iters=4, coarse_m=16, coarse_cycles=1, i_schwarz=2,
                    i_domain=4, storage_prec=DD_PREC_FP16, threads_per_site=0, setup_mode=0):
        """Two-level multigrid set-up from n_tv canonical FP64 test vectors; returns the
        set-up's device time in seconds."""
        p = dd_mg_params(n_tv, setup_iters, coarse_m, coarse_cycles,
                         dd_sap_params(i_schwarz, i_domain, storage_prec, threads_per_site, 0), setup_mode)
        sec = C.c_double()
        self._check(lib().dd_mg_setup(self._h, _ptr(tv), where, C.byref(p), C.byref(sec)))
        return sec.value

    def dd_mg_restrict(self, inp, out):
        return self._check(lib().dd_mg_restrict(self._h, _ptr(inp), _ptr(out)))

    def dd_mg_prolong(self, inp, out):
        return self._check(lib().dd_mg_prolong(self._h, _ptr(inp), _ptr(out)))

    def dd_mg_coarse_apply(self, x, y):
        return self._check(lib().dd_mg_coarse_apply(self._h, _ptr(x), _ptr(y)))

    def dd_mg_coarse_solve(self, b, x):
        return self._check(lib().dd_mg_coarse_solve(self._h, _ptr(b), _ptr(x)))

    def dd_mg_precondition(self, inp, out, layout=DD_LAYOUT_CANONICAL):
        return self._check(lib().dd_mg_precondition(self._h, _ptr(inp), _ptr(out), layout))

    def dd_solve_mg(self, f, x, where=DD_HOST, tol=1e-10, m=16, k=0, max_iter=1000, check=True):
        p = dd_solve_params(tol, m, k, max_iter, dd_sap_params(1, 1, DD_PREC_FP16, 0, 0))
        info = dd_solve_info()
        s = lib().dd_solve_mg(self._h, _ptr(f), _ptr(x), where, C.byref(p), C.byref(info))
        if check:
            self._check(s)
        return info

    def dd_spinor_bytes(self, prec, layout):
        return lib().dd_spinor_bytes(self._h, prec, layout)

    def dd_pack_spinor(self, canon, canon_prec, internal, internal_prec):
        return self._check(lib().dd_pack_spinor(self._h, _ptr(canon), canon_prec, _ptr(internal), internal_prec))

    def dd_unpack_spinor(self, internal, internal_prec, canon, canon_prec):
        return self._check(lib().dd_unpack_spinor(self._h, _ptr(internal), internal_prec, _ptr(canon), canon_prec))

    def dd_launch_count(self):
        return lib().dd_launch_count(self._h)

    def dd_autotune(self, storage_prec=DD_PREC_FP16, i_schwarz=0, i_domain=0, threads_per_site=0, additive=0):
        """Returns (domain shape, (i_schwarz, i_domain, storage_prec, threads_per_site));
        a parameter given > 0 is kept fixed; `additive` selects the Schwarz form tuned."""
        dom = (C.c_int * 4)()
        p = dd_sap_params(i_schwarz, i_domain, storage_prec, threads_per_site, additive)
        self._check(lib().dd_autotune(self._h, storage_prec, dom, C.byref(p)))
        return tuple(dom), (p.i_schwarz, p.i_domain, p.storage_prec, p.threads_per_site)


def dd_sap_precondition_lattices(ctxs, ins, outs, i_schwarz, i_domain, storage_prec=DD_PREC_FP16, nrhs=1):
    """One Schwarz launch per half-sweep over several lattices, nrhs internal FP32 fields
    per lattice one after another."""
    n = len(ctxs)
    hs = (C.c_void_p * n)(*[c._h.value for c in ctxs])
    pi = (C.c_void_p * n)(*[_ptr(x) for x in ins])
    po = (C.c_void_p * n)(*[_ptr(x) for x in outs])
    p = dd_sap_params(i_schwarz, i_domain, storage_prec, 0)
    s = lib().dd_sap_precondition_lattices(hs, pi, po, n, int(nrhs), C.byref(p))
    if s != DD_OK:
        raise DDError(s, lib().dd_last_error(ctxs[0]._h).decode())


def dd_fp32_peak(duration_ms=2000):
    """(burst, sustained) FP32 TFLOP/s of the current device from the FFMA kernel."""
    b, s = C.c_double(), C.c_double()
    st = lib().dd_fp32_peak(int(duration_ms), C.byref(b), C.byref(s))
    if st != DD_OK:
        raise DDError(st, "dd_fp32_peak failed")
    return b.value, s.value


def dd_fp64_peak(duration_ms=1000):
    """(burst, sustained) FP64 TFLOP/s of the current device from the DFMA kernel."""
    b, s = C.c_double(), C.c_double()
    st = lib().dd_fp64_peak(int(duration_ms), C.byref(b), C.byref(s))
    if st != DD_OK:
        raise DDError(st, "dd_fp64_peak failed")
    return b.value, s.value


def dd_solve_lattices(ctxs, fs, xs, nrhs=1, where=DD_HOST, tol=1e-10, m=16, k=0, max_iter=1000, i_schwarz=16,
                      i_domain=4, check=True):
    """Lockstep solves over several lattices (FP16-storage Schwarz, one launch per
    half-sweep over all of them); fs[l] / xs[l]: nrhs canonical FP64 fields of lattice l."""
    n = len(ctxs)
    hs = (C.c_void_p * n)(*[c._h.value for c in ctxs])
    pf = (C.c_void_p * n)(*[_ptr(a) for a in fs])
    px = (C.c_void_p * n)(*[_ptr(a) for a in xs])
    p = dd_solve_params(tol, m, k, max_iter, dd_sap_params(i_schwarz, i_domain, DD_PREC_FP16, 0, 0))
    info = dd_solve_info()
    s = lib().dd_solve_lattices(hs, n, pf, px, int(nrhs), where, C.byref(p), C.byref(info))
    if check and s != DD_OK:
        raise DDError(s, lib().dd_last_error(ctxs[0]._h).decode())
    return info


def dd_load_model(n_domains_per_colour, slots):
    return lib().dd_load_model(int(n_domains_per_colour), int(slots))


def dd_deflate_host(Hbar, c, y, k):
    """Host build of the deflated-restart algebra (for checks without a GPU)."""
    m = Hbar.shape[1]
    H = np.asfortranarray(Hbar.astype(np.complex128))
    P = np.zeros((m + 1, k + 1), dtype=np.complex128, order="F")
    Hn = np.zeros((m + 1, k), dtype=np.complex128, order="F")
    cn = np.zeros(k + 1, dtype=np.complex128)
    th = np.zeros(m, dtype=np.complex128)
    cc = np.ascontiguousarray(c, dtype=np.complex128)
    yy = np.ascontiguousarray(y, dtype=np.complex128)
    s = lib().dd_deflate_host(m, k, H.ctypes.data, cc.ctypes.data, yy.ctypes.data, P.ctypes.data,
                              Hn.ctypes.data, cn.ctypes.data, th.ctypes.data)
    if s != DD_OK:
        raise DDError(s, "dd_deflate_host failed")
    return P, Hn[:k + 1], cn, th


def dd_deflate_device(Hbar, c, y, k):
    """The deflated restart's small dense step on the device (one warp), as dd_solve runs
    it; returns (P, Hn, cn, theta, kernel ms) as numpy arrays."""
    import torch
    m = Hbar.shape[1]
    dev = lambda a: torch.view_as_real(torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128))).cuda()
    H = dev(Hbar.T.copy())   # column-major
    cc, yy = dev(c), dev(y)
    P = torch.zeros(k + 1, m + 1, 2, dtype=torch.float64, device="cuda")
    Hn = torch.zeros(k, m + 1, 2, dtype=torch.float64, device="cuda")
    cn = torch.zeros(k + 1, 2, dtype=torch.float64, device="cuda")
    th = torch.zeros(m, 2, dtype=torch.float64, device="cuda")
    ms = C.c_double()
    s = lib().dd_deflate_device(m, k, H.data_ptr(), cc.data_ptr(), yy.data_ptr(), P.data_ptr(), Hn.data_ptr(),
                                cn.data_ptr(), th.data_ptr(), C.byref(ms))
    if s != DD_OK:
        raise DDError(s, "dd_deflate_device failed")
    cplx = lambda t: torch.view_as_complex(t.cpu()).numpy()
    return cplx(P).T, cplx(Hn).T[:k + 1], cplx(cn), cplx(th), ms.value
