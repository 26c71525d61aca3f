"""Benchmark: time-to-solution of the mixed-precision SAP-FGMRES-DR solver on the
32^3x64 Wilson-clover workload (one GB300), with the plain-FP32 form, the full
Wilson-clover operator's bandwidth and the Schwarz kernel's FP32 rate beside it.

A step is one full solve A x = f to |f - A x| / |f| <= 1e-10 (FP64-recomputed), from
x = 0, with the gauge field, clover and source already resident in HBM.  Set-up
(gauge load, clover build) is timed separately.  Every field of this workload
(0.2-1.2 GB) is larger than the 129 MB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "32^3x64"
SAP_DTYPE = {"fp16": "f16-storage/f32-arith/f64-residual",
             "half2": "f16-storage/f16x2-products+f32-arith/f64-residual"}
SAP_KERNEL = {"fp16": "sap_kernel (Schwarz half-sweep, FP16 storage)",
              "half2": "sap_kernel (Schwarz half-sweep, FP16 storage, packed FP16 products)"}
METRIC = "time-to-solution to 1e-10 true residual, mixed FP16/FP32/FP64 SAP-FGMRES-DR"
FLOP_HOP, FLOP_CLOVER, FLOP_A = 168, 504, 1848      # Sec. II-B: 1344 = 8 x 168, 504, 1848
# Outer iterations the 32^3x64 solve takes (measured on the GPU, mixed and FP32 alike);
# only used to scale the oracle's sampled cost to a whole solve.
ORACLE_ITERS_32x64 = 696


# ------------------------------------------------------------------ flop / byte model
def sap_visit_flops(b, i_domain):
    """Useful FP32 flops per site for one domain visit of the Schwarz kernel.

    Hops that cross the domain face do not exist in the domain operator, so per
    direction only the fraction (b_mu - 1)/b_mu of the 2 hops per site is counted.
    Per MR step: the hops of D_oe and D_eo (168 each), the clover block on even sites
    and its inverse on odd sites (504 per site), and 384 flops of inner products and
    updates per even site.  Preparation and odd reconstruction each cost half the
    domain's hops plus half the clover; the face coupling, face output and the
    solution update add ~ 300 flops per site on average.
    """
    inside = sum(2.0 * (bb - 1) / bb for bb in b)           # inside hops per site
    face = sum(2.0 / bb for bb in b)                           # crossing hops per site
    mr = FLOP_HOP * inside + FLOP_CLOVER + 192.0
    prep = 0.5 * FLOP_HOP * inside + 0.5 * FLOP_CLOVER + 24.0
    recon = 0.5 * FLOP_HOP * inside + 0.5 * FLOP_CLOVER + 24.0
    faces = face * (0.5 * 156 + 0.5 * 24) + face * (12 + 0.5 * 132) + 24.0 + 48.0
    useful = i_domain * mr + prep + recon + faces
    nominal = i_domain * (FLOP_A + 192.0) + FLOP_A
    return useful, nominal


def dslash_bytes_per_site(prec):
    """Algorithmic bytes of one full operator application per site: 4 links (18 reals),
    clover (72 reals), input and output spinors (24 reals each) = 192 reals; FP16
    storage adds the two 4-byte spinor norms."""
    return {"fp64": 192 * 8, "fp32": 192 * 4, "fp16": 192 * 2 + 8}[prec]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self.rows
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def src_sha(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def read_profile(name, sha):
    """Per-launch DRAM traffic from a committed ncu summary, if it was taken on the
    current kernel source (its `source_sha` line matches)."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def max_over_ranks(vals, device="cpu"):
    """Element-wise max of per-rank timings over all ranks (identity on one rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


# ------------------------------------------------------------------ oracle arm
# The oracle's cost is sampled on smaller lattices of the workload's kind (same field
# recipe, kappa, c_sw, domain shape) and scaled per site: the FP64 operator A on a 32^3x8
# slab, one Schwarz application (I_Schwarz, I_domain of the workload) on a 16^3x8 slab.
# Both are local computations, so their cost per site does not depend on the volume.
A_SAMPLE = (32, 32, 32, 8)
SAP_SAMPLE = (16, 16, 16, 8)


def host_cpu():
    """Host CPU model and core count, for the baseline's record."""
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
            for line in out.splitlines():
                if line.startswith("Model name"):
                    model = line.split(":", 1)[1].strip()
        except OSError:
            pass
    import platform
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


def sample_workload(w, dims):
    import synth
    return synth.Workload("sample", dims, w.width, w.ape_steps, w.kappa, w.csw, w.domain, w.i_schwarz, w.i_domain,
                          w.m, w.k, w.gauge_seed, w.source_seed)


def oracle_fields(w, dims):
    """(U, F, f) of a sample lattice, generated on the GPU when there is one."""
    import torch
    from oracle import wilson as W
    ws = sample_workload(w, dims)
    U, f = make_inputs(ws, "cuda" if torch.cuda.is_available() else "cpu")
    U = U.cpu().numpy()
    return U, W.field_strength(U), f


def oracle_time_A(w, fields):
    """Seconds of one FP64 oracle application of A on the A sample lattice."""
    from oracle import wilson as W
    U, F, f = fields
    t0 = time.perf_counter()
    W.apply_A(U, f, w.kappa, w.csw, F)
    return time.perf_counter() - t0


def oracle_time_sap(w):
    """Seconds of one oracle Schwarz application on the SAP sample lattice."""
    from oracle import dd as DD
    U, F, f = oracle_fields(w, SAP_SAMPLE)
    dom = DD.Domains(SAP_SAMPLE, w.domain)
    solver = DD.BlockSolver(U, F, w.kappa, w.csw, dom)
    t0 = time.perf_counter()
    DD.sap(U, F, f, w.kappa, w.csw, dom, w.i_schwarz, w.i_domain, solver=solver)
    return time.perf_counter() - t0


def _oracle_worker(job, barrier, out):
    """One process of the all-cores oracle sample: load the sample fields, then (all
    processes together, behind a barrier with a time limit) time one A and one Schwarz
    application; the result or the error goes to the queue `out`."""
    path_a, path_s, sap_dims, kappa, csw, domain, i_s, i_d = job
    try:
        from oracle import dd as DD
        from oracle import wilson as W
        a, sp = np.load(path_a), np.load(path_s)
        Ua, fa, Us, fs = a["U"], a["f"], sp["U"], sp["f"]
        Fa, Fs = W.field_strength(Ua), W.field_strength(Us)
        dom = DD.Domains(sap_dims, domain)
        solver = DD.BlockSolver(Us, Fs, kappa, csw, dom)
        barrier.wait(timeout=300)
        t0 = time.perf_counter()
        W.apply_A(Ua, fa, kappa, csw, Fa)
        t_a = time.perf_counter() - t0
        barrier.wait(timeout=300)
        t0 = time.perf_counter()
        DD.sap(Us, Fs, fs, kappa, csw, dom, i_s, i_d, solver=solver)
        out.put(("ok", t_a, time.perf_counter() - t0))
    except Exception as e:   # release the others and report
        barrier.abort()
        out.put(("error", repr(e), 0.0))


def oracle_all_cores(w, fields_a, fields_s):
    """The oracle on every host core at once: one process per core (spawned, so no forked
    CUDA state), each timing the same A and Schwarz samples concurrently.  Returns
    (cores, seconds of A, seconds of the Schwarz application), each the slowest process's.
    Raises RuntimeError if a process fails or the samples do not finish within 10 minutes."""
    import multiprocessing as mp
    import queue
    import tempfile
    n = os.cpu_count() or 1
    tmp = tempfile.mkdtemp(prefix="oracle_sample_")
    pa, ps = os.path.join(tmp, "a.npz"), os.path.join(tmp, "s.npz")
    np.savez(pa, U=fields_a[0], f=fields_a[2])
    np.savez(ps, U=fields_s[0], f=fields_s[2])
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(n), ctx.Queue()
    job = (pa, ps, tuple(fields_s[2].shape[:4][::-1]), w.kappa, w.csw, w.domain, w.i_schwarz, w.i_domain)
    procs = [ctx.Process(target=_oracle_worker, args=(job, barrier, out)) for _ in range(n)]
    res = []
    try:
        for p in procs:
            p.start()
        deadline = time.time() + 600
        for _ in range(n):
            res.append(out.get(timeout=max(1.0, deadline - time.time())))
    except queue.Empty:
        raise RuntimeError("oracle processes did not finish within 10 minutes")
    finally:
        for p in procs:
            p.join(timeout=10)
            if p.is_alive():
                p.kill()
        for p in (pa, ps):
            os.remove(p)
        os.rmdir(tmp)
    bad = [r for r in res if r[0] != "ok"]
    if bad:
        raise RuntimeError(f"oracle process failed: {bad[0][1]}")
    return n, max(r[1] for r in res), max(r[2] for r in res)


def oracle_solve_estimate(w, t_a, t_sap, iters, reliable):
    """Oracle seconds for the whole solve: per outer iteration one A and one Schwarz
    application, plus the FP64 residuals, each scaled per site to the workload's volume."""
    V = float(np.prod(w.dims))
    a_site = t_a / float(np.prod(A_SAMPLE))
    sap_site = t_sap / float(np.prod(SAP_SAMPLE))
    return (iters * (a_site + sap_site) + reliable * a_site) * V


def a_equivalents(w, iters, reliable):
    """Operator-application equivalents of one solve: per outer iteration one A and one
    Schwarz application (I_Schwarz x 2 half-sweeps, each ~ (I_domain + 1) D
    applications on half the lattice, i.e. (I_domain + 1) / 2 A-equivalents), plus the
    FP64 residuals."""
    sap = w.i_schwarz * 2 * (w.i_domain + 1) / 2.0
    return iters * (1 + sap) + reliable


def make_inputs(w, device):
    import synth
    U = synth.make_gauge(w, device=device)
    f = synth.make_sources(w)[0]
    return U, f


def reference_arm(args):
    """The oracle as the reference arm, on the host cores: every step times one FP64 A on
    the A sample; one Schwarz application on the SAP sample is timed before the steps.
    Each step's value is the whole solve scaled from them (see oracle_solve_estimate)."""
    w = __import__("synth").WORKLOADS[WORKLOAD]
    t_sap = oracle_time_sap(w)
    fields = oracle_fields(w, A_SAMPLE)
    vals, ts = [], []
    for i in range(args.warmup + args.steps):
        t = oracle_time_A(w, fields)
        if i >= args.warmup:
            ts.append(t)
            vals.append(oracle_solve_estimate(w, t, t_sap, ORACLE_ITERS_32x64, 22))
    val = statistics.median(vals)
    cpu = host_cpu()
    sample = (f"FP64 oracle (numpy, one thread; host {cpu['model']}, {cpu['nproc']} cores): A on a "
              f"{'x'.join(map(str, A_SAMPLE))} slab (median {1e3 * statistics.median(ts):.0f} ms per step) and one "
              f"Schwarz application on a {'x'.join(map(str, SAP_SAMPLE))} slab ({t_sap:.1f} s), scaled per site to "
              f"{WORKLOAD} and to a {ORACLE_ITERS_32x64}-iteration solve with 22 FP64 residuals")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(ts),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_dict(w),
           "cpu_baseline": {"value": val, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample,
                            "host": cpu},
           "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def config_dict(w):
    return {"workload": f"{WORKLOAD} Wilson-clover, random SU(3) width {w.width} + {w.ape_steps} APE, "
                        f"kappa {w.kappa}, c_sw {w.csw}, 1 Gaussian source",
            "lattice": list(w.dims), "domain": list(w.domain), "i_schwarz": w.i_schwarz, "i_domain": w.i_domain,
            "fgmres_m": w.m, "fgmres_k": w.k, "tol": w.tol, "l2": "inputs larger than L2 (no flush)"}


# ------------------------------------------------------------------ our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-mixed", action="store_true", help="time the mixed solve only (profiling runs)")
    ap.add_argument("--case", default="solve",
                    choices=["solve", "sap", "dslash", "sap_lattices", "workload_solve", "bicgstab",
                             "lattices_solve", "lowmode", "mg"],
                    help="sap / dslash: time one kernel alone on --lattice (kernel studies, ncu captures)")
    ap.add_argument("--lattice", default="32,32,32,64")
    ap.add_argument("--domain", default="", help="kernel studies: domain shape (default: the workload's)")
    ap.add_argument("--tps", type=int, default=0, help="Schwarz kernel threads per site (0: library default)")
    ap.add_argument("--nrhs", type=int, default=1, help="kernel studies: right-hand sides per launch")
    ap.add_argument("--workload", default="48^3x96", help="workload_solve: the workload to solve once")
    ap.add_argument("--sap-prec", default="fp16", choices=["fp16", "half2"],
                    help="mixed form: FP16 storage with FP32 arithmetic, or with packed FP16 products")
    ap.add_argument("--m", type=int, default=0, help="workload_solve: basis size (0: the workload's)")
    ap.add_argument("--kappa", type=float, default=0.0, help="bicgstab: kappa (0: the workload's)")
    ap.add_argument("--max-iter", type=int, default=4000, help="bicgstab: BiCGstab iterations allowed")
    ap.add_argument("--mg-ntv", type=int, default=8, help="mg: test vectors")
    ap.add_argument("--mg-setup-iters", type=int, default=4, help="mg: Schwarz applications per test vector")
    ap.add_argument("--mg-coarse-m", type=int, default=16, help="mg: GMRES steps per coarse cycle")
    ap.add_argument("--mg-cycles", type=int, default=1, help="mg: coarse GMRES cycles")
    ap.add_argument("--mg-smooth", type=int, default=0, help="mg: smoother Schwarz cycles (0: the workload's)")
    ap.add_argument("--mg-setup-mode", type=int, default=0, help="mg: 0 v <- M v, 1 v <- v - M A v")
    ap.add_argument("--mg-m", type=int, default=16, help="mg: outer basis size")
    ap.add_argument("--mg-k", type=int, default=4, help="mg: outer deflation vectors")
    args = ap.parse_args()
    if not args.only_mixed:
        args.warmup = max(args.warmup, 3)   # profiling runs (--only-mixed) may skip the warm-up

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        if world > 1:
            dist.destroy_process_group()
        return

    import synth
    from paper_1412_2629_gb300 import build as B
    B.build()
    from paper_1412_2629_gb300 import dd
    if args.case == "sap_lattices":
        return lattices_case(args)
    if args.case == "workload_solve":
        return workload_case(args)
    if args.case == "bicgstab":
        return bicgstab_case(args)
    if args.case == "lattices_solve":
        return lattices_solve_case(args)
    if args.case == "lowmode":
        return lowmode_case(args)
    if args.case == "mg":
        return mg_case(args)
    if args.case != "solve":
        return kernel_case(args, local)

    torch.cuda.set_device(local)
    w = synth.WORKLOADS[WORKLOAD]
    st = torch.cuda.current_stream()
    U, f = make_inputs(w, "cuda")
    ctx = dd.Context(w.dims, w.domain, True, st.cuda_stream)
    t0 = time.perf_counter()
    ctx.dd_load_gauge(torch.view_as_real(U).contiguous(), dd.DD_DEVICE)
    ctx.dd_build_clover(w.kappa, w.csw)
    setup_s = time.perf_counter() - t0
    del U
    ft = torch.view_as_real(torch.from_numpy(f)).contiguous()
    f_dev = ft.to("cuda")
    x_dev = torch.zeros_like(f_dev)
    f_pin = ft.pin_memory()
    x_pin = torch.zeros_like(ft).pin_memory()
    kw = dict(tol=w.tol, m=w.m, k=w.k, i_schwarz=w.i_schwarz, i_domain=w.i_domain, max_iter=2000)

    def solve(prec, where=dd.DD_DEVICE, basis16=0):
        if where == dd.DD_DEVICE:
            x_dev.zero_()
            return ctx.dd_solve(f_dev, x_dev, where=dd.DD_DEVICE, storage_prec=prec, basis_fp16=basis16, **kw)
        x_pin.zero_()
        return ctx.dd_solve(f_pin, x_pin, where=dd.DD_HOST, storage_prec=prec, basis_fp16=basis16, **kw)

    def timed(prec, where, steps, warmup, tag, basis16=0):
        for _ in range(warmup):
            solve(prec, where, basis16)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = ctx.dd_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        torch.cuda.nvtx.range_push(tag)
        e0.record(st)
        for _ in range(steps):
            infos.append(solve(prec, where, basis16).as_dict())
        e1.record(st)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if world > 1:
            dist.barrier()
        ms = e0.elapsed_time(e1) / steps
        return ms, infos, ctx.dd_launch_count() - l0

    # FP32 CUDA-core peak, measured (FFMA microbenchmark, ~2 s of back-to-back launches)
    clk_p = ClockSampler(local)
    clk_p.start()
    peak_burst, peak_sust = dd.dd_fp32_peak(2000)
    peak_clocks = clk_p.stop()

    clk = ClockSampler(local)
    clk.start()
    mixed = dd.DD_PREC_FP16_H2 if args.sap_prec == "half2" else dd.DD_PREC_FP16
    ms_mixed, infos, launches = timed(mixed, dd.DD_DEVICE, args.steps, args.warmup, "timed_mixed")
    clocks = clk.stop()
    if args.only_mixed:
        ms_e2e, ms_fp32, infos32 = float("nan"), float("nan"), infos
        ms_alt, infos_alt = float("nan"), infos
        ms_b16, infos_b16 = float("nan"), infos
    else:
        ms_e2e, infos_e2e, _ = timed(mixed, dd.DD_HOST, args.steps, 1, "timed_e2e")
        ms_fp32, infos32, _ = timed(dd.DD_PREC_FP32, dd.DD_DEVICE, max(2, args.steps // 2), 1, "timed_fp32")
        # the other mixed form: FP16 storage with packed FP16 products (or FP32 arithmetic)
        alt = dd.DD_PREC_FP16 if args.sap_prec == "half2" else dd.DD_PREC_FP16_H2
        ms_alt, infos_alt, _ = timed(alt, dd.DD_DEVICE, max(2, args.steps // 2), 1, "timed_alt")
        # the same mixed solve with its Krylov basis stored in FP16 (beyond the paper)
        ms_b16, infos_b16, _ = timed(mixed, dd.DD_DEVICE, max(2, args.steps // 2), 1, "timed_b16", basis16=1)

    ms_mixed, ms_e2e, ms_fp32, ms_alt, ms_b16 = max_over_ranks([ms_mixed, ms_e2e, ms_fp32, ms_alt, ms_b16], "cuda")

    # the FP64 operator of the reliable update (once per restart, in "other"): timed alone on
    # the workload's fields against the measured DFMA rate; reported beside the line, never
    # allowed to stop it
    fp64_op = None
    if not args.only_mixed:
        try:
            p64_burst, p64_sust = dd.dd_fp64_peak(1000)
            a64 = torch.randn(int(np.prod(w.dims)) * 24, dtype=torch.float64, device="cuda")
            b64 = torch.empty_like(a64)
            ctx.dd_apply_D(a64, b64, dd.DD_PREC_FP64, dd.DD_LAYOUT_INTERNAL)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(st)
            for _ in range(5):
                ctx.dd_apply_D(a64, b64, dd.DD_PREC_FP64, dd.DD_LAYOUT_INTERNAL)
            ev1.record(st)
            torch.cuda.synchronize()
            ms64 = ev0.elapsed_time(ev1) / 5
            tf64 = FLOP_A * float(np.prod(w.dims)) / (ms64 * 1e-3) / 1e12
            fp64_op = {"kernel": "apply_A_kernel<double>", "bound": "fp64", "launch_ms": ms64,
                       "achieved": tf64, "peak": p64_sust, "unit": "TFLOP/s", "frac": tf64 / p64_sust,
                       "peak_note": f"of measured: DFMA microbenchmark (dd_fp64_peak), sustained over ~1 s; "
                                    f"burst {p64_burst:.2f} TFLOP/s; 1848 flop/site (Sec. II-B); each call "
                                    "includes one stream synchronisation"}
            del a64, b64
        except Exception as e:   # a missing measurement must not cost the benchmark line
            fp64_op = {"unavailable": repr(e)}

    V = int(np.prod(w.dims))
    mean = lambda key, L: statistics.mean(i[key] for i in L)
    iters = mean("iterations", infos)
    t_M, t_A, t_GS, t_other = (mean(k, infos) for k in ("t_M", "t_A", "t_GS", "t_other"))
    # Schwarz kernel: every launch is one half-sweep over the V/2 sites of one colour
    n_sap = iters * 2 * w.i_schwarz
    sap_launch_s = t_M / n_sap
    useful, nominal = sap_visit_flops(w.domain, w.i_domain)
    sap_flops_launch = useful * V / 2
    sap_tflops = sap_flops_launch / sap_launch_s / 1e12
    props = torch.cuda.get_device_properties(local)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_units = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    # the Schwarz kernel runs inside a seconds-long solve: the sustained FFMA figure
    fp32_peak = peak_sust
    sap_sha = src_sha(["paper_1412_2629_gb300/csrc/sap.cu", "paper_1412_2629_gb300/csrc/dd_common.cuh"])
    dsl_sha = src_sha(["paper_1412_2629_gb300/csrc/dslash.cu", "paper_1412_2629_gb300/csrc/dd_common.cuh"])
    sap_traffic = read_profile("sap_kernel_32x64.txt", sap_sha)
    # full operator inside the solve: one FP32 application per outer iteration
    a_launch_s = t_A / iters
    hbm = peaks.get("hbm_gbs", 6800.0)
    dsl_gbs = dslash_bytes_per_site("fp32") * V / a_launch_s / 1e9
    dsl_traffic = read_profile("dslash_fp32_32x64.txt", dsl_sha)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        fa = oracle_fields(w, A_SAMPLE)
        t_a = oracle_time_A(w, fa)
        t_sap = oracle_time_sap(w)
        rel_up = mean("reliable_updates", infos)
        host = host_cpu()
        one = oracle_solve_estimate(w, t_a, t_sap, iters, rel_up)
        # all cores: every process runs the same samples at once; n of them finish n samples
        try:
            n, ta_n, ts_n = oracle_all_cores(w, fa, oracle_fields(w, SAP_SAMPLE))
        except RuntimeError as e:
            n, ta_n, ts_n = 1, t_a, t_sap
            print(f"all-cores oracle sample unavailable ({e}); one thread reported", file=sys.stderr)
        alln = oracle_solve_estimate(w, ta_n / n, ts_n / n, iters, rel_up)
        cpu = {"value": alln, "unit": "s", "cores": n, "kind": "oracle", "host": host,
               "sample": f"FP64 oracle (numpy) on {n} processes at once (host {host['model']}, {host['nproc']} "
                         f"cores), each timing A on a {'x'.join(map(str, A_SAMPLE))} slab ({ta_n:.2f} s) and one "
                         f"Schwarz application on a {'x'.join(map(str, SAP_SAMPLE))} slab ({ts_n:.1f} s) "
                         f"concurrently; the slowest process's time / {n}, scaled per site to {WORKLOAD} and to "
                         f"this solve's {iters:.0f} iterations and {rel_up:.0f} FP64 residuals",
               "one_thread": {"value": one, "cores": 1, "a_s": t_a, "sap_s": t_sap}}

    value = ms_mixed / 1e3
    out = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": SAP_DTYPE[args.sap_prec], "data": "synthetic",
        "config": config_dict(w),
        "e2e": {"value": ms_e2e / 1e3, "unit": "s", "h2d_bytes_per_step": 2 * V * 24 * 8,
                "d2h_bytes_per_step": V * 24 * 8},
        "roofline": {"kernel": SAP_KERNEL[args.sap_prec], "bound": "alu",
                     "achieved": sap_tflops, "peak": fp32_peak, "unit": "TFLOP/s", "frac": sap_tflops / fp32_peak,
                     "traffic": sap_traffic,
                     "peak_note": "of measured: FFMA microbenchmark (dd_fp32_peak), sustained over ~2 s; "
                                  f"burst {peak_burst:.1f} TFLOP/s; unit counts {props.multi_processor_count} SMs x "
                                  f"128 lanes x 2 flop x {sm_max:.0f} MHz = {fp32_units:.1f} TFLOP/s",
                     "frac_of_unit_count_peak": sap_tflops / fp32_units,
                     "peak_clocks": peak_clocks,
                     "flops_per_launch": sap_flops_launch, "launch_ms": 1e3 * sap_launch_s},
        "dslash": {"kernel": fp32_operator_kernel(w.domain), "bound": "hbm", "achieved": dsl_gbs, "peak": hbm,
                   "unit": "GB/s", "frac": dsl_gbs / hbm, "traffic": dsl_traffic, "launch_ms": 1e3 * a_launch_s,
                   "bytes_per_launch": dslash_bytes_per_site("fp32") * V, "peak_note": "of measured (MEASURED_PEAKS hbm_gbs)"},
        ("fp16_f32arith_form" if args.sap_prec == "half2" else "half2_form"): {
            "value": ms_alt / 1e3, "unit": "s", "dtype": SAP_DTYPE["fp16" if args.sap_prec == "half2" else "half2"],
            "iterations": mean("iterations", infos_alt),
            "true_rel_residual": max(i["true_rel_residual"] for i in infos_alt),
            "schwarz_launch_ms": 1e3 * mean("t_M", infos_alt) / (mean("iterations", infos_alt) * 2 * w.i_schwarz)},
        "fp64_operator": fp64_op,
        "fp16_basis_form": {"value": ms_b16 / 1e3, "unit": "s", "iterations": mean("iterations", infos_b16),
                            "true_rel_residual": max(i["true_rel_residual"] for i in infos_b16),
                            "split_s": {"A": mean("t_A", infos_b16), "M": mean("t_M", infos_b16),
                                        "GS": mean("t_GS", infos_b16), "other": mean("t_other", infos_b16)},
                            "note": "Krylov basis V stored in FP16 (one power-of-two scale), everything else "
                                    "as the headline solve; beyond the paper"},
        "fp32_form": {"value": ms_fp32 / 1e3, "unit": "s", "iterations": mean("iterations", infos32),
                      "true_rel_residual": max(i["true_rel_residual"] for i in infos32),
                      "speedup_mixed_over_fp32": ms_fp32 / ms_mixed},
        "solve": {"iterations": iters, "restarts": mean("restarts", infos),
                  "deflated_restarts": mean("deflated_restarts", infos),
                  "reliable_updates": mean("reliable_updates", infos),
                  "true_rel_residual": max(i["true_rel_residual"] for i in infos),
                  "split_s": {"A": t_A, "M": t_M, "GS": t_GS, "other": t_other},
                  "sap_gflops_nominal": nominal * V / 2 / sap_launch_s / 1e9,
                  "setup_s": setup_s},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if cpu is not None:
        out["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def kernel_case(args, local):
    """Time one kernel alone (Schwarz half-sweeps or the FP32 operator) on a lattice of
    the 32^3x64 workload's kind, with CUDA events on the launching stream."""
    import torch

    import synth
    from paper_1412_2629_gb300 import dd
    SAP_PREC = {"fp16": dd.DD_PREC_FP16, "half2": dd.DD_PREC_FP16_H2}
    base = synth.WORKLOADS[WORKLOAD]
    dims = tuple(int(v) for v in args.lattice.split(","))
    dom = tuple(int(v) for v in args.domain.split(",")) if args.domain else base.domain
    w = synth.Workload("case", dims, base.width, base.ape_steps, base.kappa, base.csw, dom, base.i_schwarz,
                       base.i_domain, base.m, base.k, base.gauge_seed, base.source_seed)
    st = torch.cuda.current_stream()
    U, f = make_inputs(w, "cuda")
    ctx = dd.Context(w.dims, w.domain, True, st.cuda_stream)
    ctx.dd_load_gauge(torch.view_as_real(U).contiguous(), dd.DD_DEVICE)
    ctx.dd_build_clover(w.kappa, w.csw)
    del U
    V = int(np.prod(dims))
    src = torch.view_as_real(torch.from_numpy(f)).to(torch.float32).cuda().contiguous()
    nb = ctx.dd_spinor_bytes(dd.DD_PREC_FP32, dd.DD_LAYOUT_INTERNAL)
    nr = args.nrhs
    a = torch.empty(nr * nb, dtype=torch.uint8, device="cuda")
    b = torch.empty_like(a)
    for r in range(nr):
        ctx.dd_pack_spinor(src, dd.DD_PREC_FP32, a[r * nb:(r + 1) * nb], dd.DD_PREC_FP32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = args.steps
    if args.case == "sap" and nr > 1:
        run = lambda: ctx.dd_sap_precondition_batch(a, b, nr, w.i_schwarz, w.i_domain, SAP_PREC[args.sap_prec])
        launches = 2 * w.i_schwarz
    elif args.case == "sap":
        run = lambda: ctx.dd_sap_precondition(a, b, w.i_schwarz, w.i_domain, SAP_PREC[args.sap_prec], dd.DD_LAYOUT_INTERNAL,
                                              threads_per_site=args.tps)
        launches = 2 * w.i_schwarz
    elif nr > 1:
        run = lambda: ctx.dd_apply_D_batch(a, b, nr, dd.DD_PREC_FP32)
        launches = 1
    else:
        run = lambda: ctx.dd_apply_D(a, b, dd.DD_PREC_FP32, dd.DD_LAYOUT_INTERNAL)
        launches = 1
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        run()
    e1.record(st)
    torch.cuda.synchronize()
    launch_s = e0.elapsed_time(e1) / 1e3 / (reps * launches)
    if args.case == "sap":
        useful, nominal = sap_visit_flops(w.domain, w.i_domain)
        out = {"case": "sap_kernel", "threads_per_site": args.tps or 2, "nrhs": nr, "lattice": dims,
               "launch_ms": 1e3 * launch_s, "tflops_useful": nr * useful * V / 2 / launch_s / 1e12,
               "gflops_nominal": nr * nominal * V / 2 / launch_s / 1e9}
    else:
        # per right-hand side the batch reads the links and clover once per pair
        per_site = dslash_bytes_per_site("fp32") if nr == 1 else (72 + 72) * 4 / 2 + 48 * 4
        out = {"case": fp32_operator_kernel(w.domain) if nr == 1 else "apply_A_multi_kernel<float,2>", "nrhs": nr,
               "lattice": dims, "launch_ms": 1e3 * launch_s,
               "ms_per_rhs": 1e3 * launch_s / nr,
               "gbs_algorithmic": per_site * V * nr / launch_s / 1e9}
    print(json.dumps(out))


def fp32_operator_kernel(domain):
    """Name of the FP32 operator kernel the library launches for this domain shape: the
    8x4x4x4 and 4x4x4x4 shapes have compile-time specialisations."""
    shape = {(8, 4, 4, 4): 1, (4, 4, 4, 4): 2}.get(tuple(domain), 0)
    return f"apply_A_shape_kernel<{shape}>" if shape else "apply_A_kernel<float>"


def lattices_case(args):
    """The uneven batch of the fifth workload: 16^3x32, 24^3x48 and 32^3x64 (kappa 0.134,
    0.135, 0.1355, c_sw 1.5, 4^4 domains) with --nrhs Gaussian sources each (the workload
    states 8), one Schwarz application of every source, timed as one launch per half-sweep
    over all three lattices and as three separate batched calls."""
    import torch

    import synth
    from paper_1412_2629_gb300 import dd
    base = synth.WORKLOADS[WORKLOAD]
    st = torch.cuda.current_stream()
    specs = [((16, 16, 16, 32), 0.1340, 151), ((24, 24, 24, 48), 0.1350, 152), ((32, 32, 32, 64), 0.1355, 153)]
    ctxs, ins, outs, vols = [], [], [], []
    for dims, kappa, seed in specs:
        w = synth.Workload("lat", dims, base.width, base.ape_steps, kappa, 1.5, (4, 4, 4, 4), base.i_schwarz,
                           base.i_domain, base.m, base.k, seed, seed + 10)
        U, f = make_inputs(w, "cuda")
        c = dd.Context(dims, (4, 4, 4, 4), True, st.cuda_stream)
        c.dd_load_gauge(torch.view_as_real(U).contiguous(), dd.DD_DEVICE)
        c.dd_build_clover(kappa, 1.5)
        del U
        nb = c.dd_spinor_bytes(dd.DD_PREC_FP32, dd.DD_LAYOUT_INTERNAL)
        nr = args.nrhs
        a = torch.empty(nr * nb, dtype=torch.uint8, device="cuda")
        for r in range(nr):
            fr = f if r == 0 else synth.gaussian_source(dims, seed + 10 + r)
            c.dd_pack_spinor(torch.view_as_real(torch.from_numpy(fr)).float().cuda().contiguous(), dd.DD_PREC_FP32,
                             a[r * nb:(r + 1) * nb], dd.DD_PREC_FP32)
        ctxs.append(c); ins.append(a); outs.append(torch.empty_like(a)); vols.append(int(np.prod(dims)))
    i_s, i_d, nr = base.i_schwarz, base.i_domain, args.nrhs
    one = lambda: dd.dd_sap_precondition_lattices(ctxs, ins, outs, i_s, i_d, nrhs=nr)
    sep = lambda: [c.dd_sap_precondition_batch(a, o, nr, i_s, i_d, dd.DD_PREC_FP16)
                   for c, a, o in zip(ctxs, ins, outs)]
    res = {}
    for name, fn in (("one_launch", one), ("separate", sep)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        res[name + "_ms"] = e0.elapsed_time(e1) / args.steps
    useful, _ = sap_visit_flops((4, 4, 4, 4), i_d)
    res["tflops_one_launch"] = useful * sum(vols) * i_s * nr / (res["one_launch_ms"] / 1e3) / 1e12
    res["case"] = "sap_lattices 16^3x32 + 24^3x48 + 32^3x64"
    res["nrhs_per_lattice"] = nr
    print(json.dumps(res))


def workload_case(args):
    """One mixed-precision solve of a named workload (the larger lattices: 48^3x96,
    64^3x128), device-resident f and x, with the times of input generation, set-up and
    solve; the true residual is the library's FP64 recomputation.  With --nrhs N > 1
    (the batched 24^3x48 workload: 12 point sources, then Gaussian ones) the N solves run
    in lockstep and, for comparison, one after another."""
    import torch

    import synth
    from paper_1412_2629_gb300 import dd
    w = synth.WORKLOADS[args.workload]
    st = torch.cuda.current_stream()
    t0 = time.perf_counter()
    U = synth.random_su3_field(w.dims, w.width, w.gauge_seed, device="cuda")
    torch.cuda.synchronize()
    t_rand = time.perf_counter() - t0
    if w.ape_steps:
        U = synth.ape_smear(U, 0.5, w.ape_steps)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    nr = args.nrhs
    if nr > 1:   # the batched workload's mix: the 12 point sources first, then Gaussian ones
        pts = synth.point_sources(w.dims)
        fs = pts[:min(nr, 12)] + synth.make_sources(w, max(0, nr - 12))
        f = np.stack(fs)
        del pts, fs
    else:
        f = synth.make_sources(w)[0]
    ctx = dd.Context(w.dims, w.domain, True, st.cuda_stream)
    t1 = time.perf_counter()
    ctx.dd_load_gauge(torch.view_as_real(U).contiguous(), dd.DD_DEVICE)
    ctx.dd_build_clover(w.kappa, w.csw)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t1
    del U
    torch.cuda.empty_cache()   # the generator's temporaries, before the solver allocates its basis
    f_dev = torch.view_as_real(torch.from_numpy(f)).cuda().contiguous()
    del f
    x_dev = torch.zeros_like(f_dev)
    m = args.m or w.m
    kw = dict(tol=w.tol, m=m, k=w.k, max_iter=20000, i_schwarz=w.i_schwarz, i_domain=w.i_domain)

    def run():
        x_dev.zero_()
        t = time.perf_counter()
        info = ctx.dd_solve(f_dev, x_dev, nrhs=nr, where=dd.DD_DEVICE, **kw)
        return info, time.perf_counter() - t

    out = {"case": "workload_solve", "workload": w.name, "lattice": list(w.dims), "kappa": w.kappa, "csw": w.csw,
           "domain": list(w.domain), "i_schwarz": w.i_schwarz, "i_domain": w.i_domain, "m": m, "k": w.k,
           "nrhs": nr, "gen_random_s": t_rand, "gen_total_s": t_gen, "setup_s": t_setup}
    forms = [("lockstep", "0"), ("sequential", "1")] if nr > 1 else [("single", "0")]
    for name, seq in forms:
        os.environ["DD_SEQUENTIAL_RHS"] = seq
        if nr > 1:
            run()   # warm-up: allocations and first launches
        info, wall = run()
        out[name] = {"iterations": info.iterations, "restarts": info.restarts,
                     "true_rel_residual": info.true_rel_residual, "solve_s": info.t_total, "wall_s": wall,
                     "split_s": {"A": info.t_A, "M": info.t_M, "GS": info.t_GS, "other": info.t_other}}
    os.environ.pop("DD_SEQUENTIAL_RHS", None)
    out["device_gb_in_use"] = (lambda fr: (fr[1] - fr[0]) / 1e9)(torch.cuda.mem_get_info())
    print(json.dumps(out))


def lattices_solve_case(args):
    """The uneven batch of the fifth workload solved: 16^3x32 (kappa 0.134), 24^3x48
    (0.135) and 32^3x64 (0.1355), c_sw 1.5, --nrhs Gaussian sources each (the workload
    states 8), 4^4 domains (24 / 8 is odd), in lockstep with one Schwarz launch per
    half-sweep over all three lattices (dd_solve_lattices), and, for comparison, one
    lattice after another (dd_solve with its lockstep over that lattice's sources).
    Domains 4x4x4x8 (512 sites, the volume of the 32^3x64 workload's 8x4x4x4; 24 / 8 is odd
    in space, 48 / 8 is even in time) and the settings that converge on that supercritical
    workload: I_S 2, I_d 4, k 8; --m sets the basis (default 32: the 24 solves' bases then
    take ~170 GB); at most --max-iter steps per source."""
    import torch

    import synth
    from paper_1412_2629_gb300 import dd
    base = synth.WORKLOADS[WORKLOAD]
    st = torch.cuda.current_stream()
    specs = [((16, 16, 16, 32), 0.1340, 151), ((24, 24, 24, 48), 0.1350, 152), ((32, 32, 32, 64), 0.1355, 153)]
    nr, m = args.nrhs, args.m or 32
    dom = (4, 4, 4, 8)
    kw = dict(tol=1e-10, m=m, k=8, max_iter=args.max_iter, i_schwarz=2, i_domain=4)
    ctxs, fs, xs = [], [], []
    for dims, kappa, seed in specs:
        w = synth.Workload("lat", dims, base.width, base.ape_steps, kappa, 1.5, dom, 2, 4, m, 8, seed, seed + 10)
        U = synth.make_gauge(w, device="cuda")
        c = dd.Context(dims, dom, True, st.cuda_stream)
        c.dd_load_gauge(torch.view_as_real(U).contiguous(), dd.DD_DEVICE)
        c.dd_build_clover(kappa, 1.5)
        del U
        f = np.stack(synth.make_sources(w, nr))
        fs.append(torch.view_as_real(torch.from_numpy(f)).cuda().contiguous())
        xs.append(torch.zeros_like(fs[-1]))
        ctxs.append(c)
    torch.cuda.empty_cache()
    out = {"case": "lattices_solve", "lattices": [list(d) for d, _, _ in specs], "kappa": [k for _, k, _ in specs],
           "nrhs_per_lattice": nr, "domain": list(dom), "m": m, "k": 8, "i_schwarz": 2, "i_domain": 4,
           "max_iter": args.max_iter}
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    info = dd.dd_solve_lattices(ctxs, fs, xs, nrhs=nr, where=dd.DD_DEVICE, check=False, **kw)
    out["one_launch"] = {"status": info.status, "iterations": info.iterations, "solve_s": info.t_total,
                         "true_rel_residual": info.true_rel_residual,
                         "split_s": {"A": info.t_A, "M": info.t_M, "GS": info.t_GS, "other": info.t_other}}
    tot, worst, its = 0.0, 0.0, 0
    for c, f, x in zip(ctxs, fs, xs):
        x.zero_()
        i1 = c.dd_solve(f, x, nrhs=nr, where=dd.DD_DEVICE, check=False, **kw)
        tot += i1.t_total
        worst = max(worst, i1.true_rel_residual)
        its += i1.iterations
    out["per_lattice"] = {"iterations": its, "solve_s": tot, "true_rel_residual": worst}
    out["device_gb_in_use"] = (lambda fr: (fr[1] - fr[0]) / 1e9)(torch.cuda.mem_get_info())
    print(json.dumps(out))


def lowmode_case(args):
    """The smallest |eigenvalue| of the Hermitian gamma5 A of a workload (48^3x96 by
    default), which the near-critical workload asks to be about 1e-3: power iteration on
    (gamma5 A)^-2 = (A^dag A)^-1, each step two solves of A (dd_solve, mixed form, the
    workload's parameters) with gamma5 between them; the Rayleigh quotient after --steps
    iterations bounds min |lambda(gamma5 A)| from above.  The free-field value at the same
    mass, antiperiodic time, is reported beside it."""
    import torch

    import synth
    from paper_1412_2629_gb300 import dd
    w = synth.WORKLOADS[args.workload]
    kappa = args.kappa or w.kappa
    st = torch.cuda.current_stream()
    U = synth.make_gauge(w, device="cuda")
    ctx = dd.Context(w.dims, w.domain, True, st.cuda_stream)
    ctx.dd_load_gauge(torch.view_as_real(U).contiguous(), dd.DD_DEVICE)
    ctx.dd_build_clover(kappa, w.csw)
    del U
    torch.cuda.empty_cache()
    g5 = torch.tensor([1.0, 1.0, -1.0, -1.0], dtype=torch.float64, device="cuda").view(4, 1, 1)
    x = torch.view_as_real(torch.from_numpy(synth.make_sources(w)[0])).cuda().contiguous()
    x /= x.norm()
    kw = dict(where=dd.DD_DEVICE, tol=1e-9, m=w.m, k=w.k, max_iter=20000, i_schwarz=w.i_schwarz,
              i_domain=w.i_domain)
    hist, iters, t0 = [], 0, time.perf_counter()
    for _ in range(args.steps):
        y = torch.zeros_like(x)
        iters += ctx.dd_solve((g5 * x).contiguous(), y, **kw).iterations      # y = A^-1 g5 x
        z = torch.zeros_like(x)
        iters += ctx.dd_solve((g5 * y).contiguous(), z, **kw).iterations      # z = A^-1 g5 y
        rq = float((x * z).sum())                                              # <x, (A^dag A)^-1 x>, |x| = 1
        hist.append(1.0 / math.sqrt(rq))
        x = z / z.norm()
    L = w.dims
    m0 = 1.0 / (2.0 * kappa) - 4.0
    # free field: A(p) = m0 + sum(1 - cos p) + i gamma.sin p, |lambda|^2 = (m0 + sum(1-cos))^2 + sum sin^2
    free = min(math.sqrt((m0 + sum(1 - math.cos(p) for p in ps)) ** 2 + sum(math.sin(p) ** 2 for p in ps))
               for ps in [(0.0, 0.0, 0.0, math.pi / L[3]), (0.0, 0.0, 0.0, -math.pi / L[3])])
    out = {"case": "lowmode", "workload": w.name, "kappa": kappa, "csw": w.csw, "power_steps": args.steps,
           "min_abs_lambda_g5A_upper_bound": hist[-1], "history": hist, "solve_iterations": iters,
           "seconds": time.perf_counter() - t0, "free_field_min_abs_lambda": free, "bare_mass": m0}
    print(json.dumps(out))


def mg_case(args):
    """The Schwarz method as the smoother of a two-level aggregation multigrid (the use of
    domain-decomposition preconditioners in the paper's related work, Sec. V) on the
    benchmark's lattice (--workload; default 32^3x64): set-up time, time-to-solution with
    FGMRES-DR around the two-level method against the benchmark's SAP-FGMRES-DR solve on the
    same source, and the multigrid kernels alone (CUDA events; HBM roofline of the
    restriction and prolongation, which stream the interpolation)."""
    import torch

    import synth
    from paper_1412_2629_gb300 import dd
    base = synth.WORKLOADS[args.workload if args.workload in synth.WORKLOADS else WORKLOAD]
    kappa = args.kappa or base.kappa
    st = torch.cuda.current_stream()
    U, f = make_inputs(base, "cuda")
    ctx = dd.Context(base.dims, base.domain, True, st.cuda_stream)
    ctx.dd_load_gauge(torch.view_as_real(U).contiguous(), dd.DD_DEVICE)
    ctx.dd_build_clover(kappa, base.csw)
    del U
    torch.cuda.empty_cache()
    ntv = args.mg_ntv
    smooth = args.mg_smooth or base.i_schwarz
    tv = torch.empty((ntv,) + tuple(base.dims[::-1]) + (4, 3, 2), dtype=torch.float64, device="cuda")
    for k in range(ntv):
        tv[k].copy_(torch.view_as_real(torch.from_numpy(synth.gaussian_source(base.dims, 1000 + k))))
    setup_s = ctx.dd_mg_setup(tv, ntv, dd.DD_DEVICE, setup_iters=args.mg_setup_iters, coarse_m=args.mg_coarse_m,
                              coarse_cycles=args.mg_cycles, i_schwarz=smooth, i_domain=base.i_domain,
                              storage_prec=dd.DD_PREC_FP16, setup_mode=args.mg_setup_mode)
    del tv
    torch.cuda.empty_cache()
    fd = torch.view_as_real(torch.from_numpy(f)).cuda().contiguous()
    xd = torch.zeros_like(fd)
    out = {"case": "mg", "workload": base.name, "kappa": kappa, "csw": base.csw, "n_tv": ntv,
           "setup_iters": args.mg_setup_iters, "setup_mode": args.mg_setup_mode, "coarse_m": args.mg_coarse_m, "coarse_cycles": args.mg_cycles,
           "smoother": {"i_schwarz": smooth, "i_domain": base.i_domain, "storage": "fp16"},
           "outer": {"m": args.mg_m, "k": args.mg_k}, "setup_s": setup_s}
    solves = []
    for rep in range(max(args.steps, 1) + 1):      # the first solve captures the step graphs
        xd.zero_()
        torch.cuda.synchronize()
        info = ctx.dd_solve_mg(fd, xd, where=dd.DD_DEVICE, tol=base.tol, m=args.mg_m, k=args.mg_k,
                               max_iter=args.max_iter, check=False)
        if rep > 0:
            solves.append(info)
    best = min(solves, key=lambda i: i.t_total)
    out["mg_solve"] = {"status": best.status, "iterations": best.iterations, "restarts": best.restarts,
                       "true_rel_residual": best.true_rel_residual, "solve_s": best.t_total,
                       "t_A_s": best.t_A, "t_M_s": best.t_M, "t_GS_s": best.t_GS,
                       "median_solve_s": statistics.median(i.t_total for i in solves)}
    ref = []
    for rep in range(2):
        xd.zero_()
        torch.cuda.synchronize()
        ref.append(ctx.dd_solve(fd, xd, where=dd.DD_DEVICE, tol=base.tol, m=base.m, k=base.k, max_iter=5000,
                                i_schwarz=base.i_schwarz, i_domain=base.i_domain, check=False))
    r = min(ref, key=lambda i: i.t_total)
    out["sap_solve"] = {"iterations": r.iterations, "true_rel_residual": r.true_rel_residual, "solve_s": r.t_total,
                        "m": base.m, "k": base.k}
    out["speedup_mg_over_sap"] = r.t_total / best.t_total
    # kernels alone
    V = int(np.prod(base.dims))
    nd = V // int(np.prod(base.domain))
    n_f = V * 24
    a = torch.randn(n_f, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    cvec = torch.randn(nd * 2 * ntv * 2, dtype=torch.float32, device="cuda")
    cout = torch.empty_like(cvec)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6782.8)
    t_r = timed(lambda: ctx.dd_mg_restrict(a, cvec))
    t_p = timed(lambda: ctx.dd_mg_prolong(cvec, b))
    t_c = timed(lambda: ctx.dd_mg_coarse_apply(cvec, cout))
    t_s = timed(lambda: ctx.dd_mg_coarse_solve(cvec, cout), reps=5)
    t_b = timed(lambda: ctx.dd_mg_precondition(a, b, dd.DD_LAYOUT_INTERNAL), reps=5)
    bytes_rp = (ntv + 1) * V * 96            # interpolation plus one FP32 field
    dc_bytes = nd * 9 * (2 * ntv) ** 2 * 8
    out["kernels"] = {
        "restrict_ms": t_r, "restrict_gbs": bytes_rp / t_r / 1e6, "prolong_ms": t_p,
        "prolong_gbs": bytes_rp / t_p / 1e6, "hbm_peak_gbs": hbm,
        "restrict_frac": bytes_rp / t_r / 1e6 / hbm, "prolong_frac": bytes_rp / t_p / 1e6 / hbm,
        "coarse_apply_ms": t_c, "coarse_operator_bytes": dc_bytes, "coarse_apply_gbs": dc_bytes / t_c / 1e6,
        "coarse_solve_ms": t_s, "precondition_ms": t_b,
        "note": "host-synchronous calls: each time includes one launch and stream synchronisation"}
    print(json.dumps(out))


def bicgstab_case(args):
    """The paper's comparison (Sec. IV-C, Table III non-DD rows) on one GPU: the standard
    solvers -- BiCGstab in FP64, and FP64 Richardson around FP32 BiCGstab -- against the
    domain-decomposed solver (mixed form, the benchmark's parameters) on the same lattice,
    source and kappa; device-resident f and x, time-to-solution with CUDA events."""
    import torch

    import synth
    from paper_1412_2629_gb300 import dd
    base = synth.WORKLOADS[args.workload if args.workload in synth.WORKLOADS else WORKLOAD]
    kappa = args.kappa or base.kappa
    st = torch.cuda.current_stream()
    U, f = make_inputs(base, "cuda")
    ctx = dd.Context(base.dims, base.domain, True, st.cuda_stream)
    ctx.dd_load_gauge(torch.view_as_real(U).contiguous(), dd.DD_DEVICE)
    ctx.dd_build_clover(kappa, base.csw)
    del U
    fd = torch.view_as_real(torch.from_numpy(f)).cuda().contiguous()
    xd = torch.zeros_like(fd)
    out = {"case": "bicgstab", "workload": base.name, "kappa": kappa, "csw": base.csw, "max_iter": args.max_iter}
    runs = [("dd_mixed", lambda: ctx.dd_solve(fd, xd, where=dd.DD_DEVICE, tol=base.tol, m=base.m, k=base.k,
                                              max_iter=5000, i_schwarz=base.i_schwarz, i_domain=base.i_domain,
                                              check=False)),
            ("bicgstab_fp64", lambda: ctx.dd_solve_bicgstab(fd, xd, where=dd.DD_DEVICE, tol=base.tol,
                                                            max_iter=args.max_iter, precision=dd.DD_PREC_FP64,
                                                            check=False)),
            ("richardson_bicgstab_fp32", lambda: ctx.dd_solve_bicgstab(fd, xd, where=dd.DD_DEVICE, tol=base.tol,
                                                                       max_iter=args.max_iter,
                                                                       precision=dd.DD_PREC_FP32, inner_tol=1e-5,
                                                                       check=False))]
    for name, fn in runs:
        xd.zero_()
        torch.cuda.synchronize()
        info = fn()
        out[name] = {"status": info.status, "iterations": info.iterations, "corrections": info.restarts + 1,
                     "true_rel_residual": info.true_rel_residual, "solve_s": info.t_total, "t_A_s": info.t_A}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
