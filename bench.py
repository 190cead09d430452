"""Benchmark: block-Jacobi PCG to relative residual 1e-10 on the 3D variable-coefficient
diffusion workload (128^3 grid, 7-point stencil, log-normal face coefficients with
sigma = 2, b ~ N(0,1) seed 0), mixed precision (FP32 block factors, FP64 CG) against
all-FP64.

One step = pcg_solve through the C ABI: the CSR structure check, block extraction + batched
block Cholesky/inverse (setup) and the CG solve (a CUDA graph with a device-driven loop) to
||r||/||b|| <= 1e-10 with the true-residual check.  The headline line also carries:

* the per-kernel breakdown and the roofline of the dominant kernel (the SpMV);
* the FP64-factor comparison and the block-size sweep (8/16/32/64);
* the Lanczos kappa estimates before and after preconditioning;
* the error of every result against the FP64 oracle's solution of the same system;
* the end-to-end figure (host buffers through the C ABI);
* the oracle's CPU baseline, single-threaded and on all host cores;
* sub-objects for the other two throughput workloads (512 uneven RGG systems in one
  persistent launch; the 8M-row power-law matrix with FP32 values), each with its own
  roofline, clocks, iterations, residuals and oracle error;
* the paper's own rows: point Jacobi (block size 1) setup + apply against the oracle, the
  error of the decoupled per-block solve x = M^-1 b, and the paper-size sweep of kappa and
  kappa^2 per block size.

Single workloads print their own line: --workload batched_rgg_512, --workload powerlaw_8m.

value   = algorithmic bytes of the step / step time (GB/s), inputs resident in HBM.
          bytes = setup (CSR read + factor writes) + per-solve extras (initial and final
          residual, final x update) + iterations * B_it, where
          B_it = CSR (val+col+row_ptr) + M^{-1} factor + 11 vector streams of 8N bytes.
e2e     = the same metric through the C ABI with host buffers: the CSR and b are copied
          from pinned host memory to the device and x back inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own replica (weak scaling); the sub-workloads,
paper rows and oracle comparisons run at N = 1 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2410_02408_gb300 import workloads as W  # noqa: E402

METRIC = "PCG+precond GB/s (% HBM peak), mixed vs FP64, to rel. residual 1e-10"
FALLBACK_HBM_GBS = 6800.0
# Launch shape of the batched workload when its autotuner is skipped (the fastest measured on
# the 512-system batch for each factor precision): CTAs per SM, team limit, slots per CTA,
# setup shared memory (KB).
BATCH_SHAPE_DEFAULT = {"fp32": "2,4,8,70", "tf32": "2,4,8,70", "fp64": "2,8,4,70"}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128, help="grid points per axis")
    ap.add_argument("--sigma", type=float, default=2.0)
    ap.add_argument("--bs", type=int, default=None, help="block size (default 16; 32 for powerlaw_8m)")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "tf32"])
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--maxit", type=int, default=200000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-oracle-error", action="store_true", help="skip the full oracle solves (error vs oracle)")
    ap.add_argument("--no-sub", action="store_true", help="headline: skip the batched and power-law sub-objects")
    ap.add_argument("--no-paper-rows", action="store_true", help="headline: skip point Jacobi, decoupled solve, sweep")
    ap.add_argument("--sub-steps", type=int, default=3, help="timed steps of each sub-workload")
    ap.add_argument("--cpu-sample-iters", type=int, default=0, help="oracle CG iterations per sample (0 = auto)")
    ap.add_argument("--cpu-threads", type=int, default=0, help="oracle threads of the all-cores baseline (0 = all)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="persistent CG CTAs per SM (0 = occupancy max)")
    ap.add_argument("--workload", default="diffusion3d", choices=["diffusion3d", "batched_rgg_512", "powerlaw_8m"],
                    help="diffusion3d: the headline 128^3 solve; batched_rgg_512: 512 uneven RGG systems "
                         "set up and solved in one persistent launch; powerlaw_8m: random SPD with power-law "
                         "rows (N = 8M, ~256M nnz, FP32 values, bs 32)")
    ap.add_argument("--pl-n", type=int, default=8_000_000, help="rows of the power-law workload")
    ap.add_argument("--no-kappa", action="store_true", help="skip the Lanczos kappa timing")
    ap.add_argument("--no-bs-sweep", action="store_true", help="skip the block-size sweep (8/16/32/64)")
    ap.add_argument("--row-binning", default="auto", choices=["auto", "on", "off"],
                    help="row order of the CG SpMV (auto: binned by length when rows are irregular)")
    ap.add_argument("--col-segments", default="auto",
                    help="column segments of the binned SpMV: auto (the library default, 1) or 1..8")
    ap.add_argument("--n-sys", type=int, default=512, help="systems in the batched workload")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the launch-shape autotuners (single-system loop kernels; batched launch)")
    ap.add_argument("--tune-trials", type=int, default=0, help="batched autotuner candidates (0 = all)")
    ap.add_argument("--batch-shape", default="",
                    help="batched workload: explicit launch shape 'ctas_per_sm,team_max,slots_per_cta,setup_kb' "
                         "(skips the autotuner)")
    ap.add_argument("--phase-profile", action="store_true",
                    help="batched workload: one extra solve with per-phase device timers (not timed)")
    ap.add_argument("--profile", action="store_true",
                    help="one solve of the workload and nothing else (for ncu captures); prints a short line")
    args = ap.parse_args(argv)
    args.bs_given = args.bs is not None
    if args.bs is None:
        args.bs = 16
    return args


def run_profile(args):
    """A single setup + solve (max_iter may cut it short) for profiler captures."""
    import torch

    import paper_2410_02408_gb300 as pc

    pc.load()
    pc.set_row_binning(args.row_binning)
    pc.set_col_segments(args.col_segments)
    if args.ctas_per_sm:
        pc.set_ctas_per_sm(args.ctas_per_sm)
    A, _, bs = single_workload(args)
    b = torch.from_numpy(W.rhs(A.n, 0)).cuda()
    Ad = pc.csr(A)
    x, info = pc.pcg(Ad, b, bs, tol=args.tol, max_iter=args.maxit, prec=args.prec, check=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile": True, "n": A.n, "bs": bs, "prec": args.prec, "iterations": info["iterations"],
                      "status": info["status"], "solve_ms": info["solve_ms"], "setup_ms": info["setup_ms"],
                      "grid_ctas": info["grid_ctas"]}))


# ---------------------------------------------------------------- byte accounting
def csr_bytes(n, nnz, val_bytes):
    return val_bytes * nnz + 4 * nnz + 4 * (n + 1)


def layout_units(n, bs):
    if bs <= 32:
        U = (32 // bs) * bs
        S = 1
    else:
        U = bs
        S = 2
    return (n + U - 1) // U, S


def factor_bytes(n, bs, fac_bytes):
    units, S = layout_units(n, bs)
    minv = units * (bs // 2 + 1) * S * 32 * fac_bytes
    linv = units * bs * S * 32 * fac_bytes
    return minv, linv


def step_bytes(n, nnz, bs, prec, iters, val_bytes=8):
    fb = 4 if prec != "fp64" else 8
    C = csr_bytes(n, nnz, val_bytes)
    Fm, Fl = factor_bytes(n, bs, fb)
    v = 8 * n
    b_it = C + Fm + 11 * v
    setup = C + Fm + Fl
    extras = 2 * C + Fm + 13 * v
    return setup + extras + iters * b_it, b_it, iters * b_it + extras


# ---------------------------------------------------------------- environment helpers
def measured_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"pc_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# Sources that define the profiled CG SpMV kernels: a recorded DRAM traffic stays valid while
# these files are unchanged (the binned one also depends on the row order and sliced copy).
SPMV_SOURCES = ("pc_cg_graph.cu", "pc_common.cuh", "pc_kernels.cuh", "pc_tma.cuh")
BIN_SPMV_SOURCES = SPMV_SOURCES + ("pc_rowbin.cu",)
TRAFFIC_PROFILES = {"diffusion3d": ("cg_spmv_kernel_diffusion3d_128.md", SPMV_SOURCES),
                    "powerlaw_8m": ("cg_spmv_bin_pipe_kernel_powerlaw_8m.md", BIN_SPMV_SOURCES)}


def kernel_source_hash(sources=SPMV_SOURCES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2410_02408_gb300", "csrc")
    for fn in sources:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per launch of the workload's SpMV kernel from the committed ncu summary, or
    None if absent or if the kernel's sources changed since it was taken."""
    name, sources = TRAFFIC_PROFILES[workload]
    path = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_hash:\s*(\w+)", txt)
    if not m or m.group(1) != kernel_source_hash(sources):
        return None
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    return float(m.group(1)) if m else None


def single_workload(args):
    """The single-system workload: (host CSR, name, block size)."""
    if args.workload == "powerlaw_8m":
        A = W.powerlaw_spd(args.pl_n, seed=5)
        return A, f"powerlaw_{args.pl_n}_fp32vals", (args.bs if args.bs_given else 32)
    A = W.diffusion3d(args.n, args.sigma)
    return A, f"diffusion3d_{args.n}_sigma{args.sigma:g}", args.bs


# ---------------------------------------------------------------- distributed plumbing
def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist

    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend=backend)
    return dist.get_rank(), ws, dist


def max_over_ranks(v, dist):
    if dist is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------- oracle (CPU) timing
def host_info():
    """Host cores and CPU model (the timing host of the CPU baseline)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
        m = re.search(r"^model name\s*:\s*(.+)$", txt, re.M)
        if m:
            model = m.group(1).strip()
        else:
            parts = [re.search(rf"^{k}\s*:\s*(\S+)", txt, re.M) for k in ("CPU implementer", "CPU part")]
            if all(parts):
                model = f"{platform.machine()} implementer {parts[0].group(1)} part {parts[1].group(1)}"
    except OSError:
        pass
    return {"nproc": cores, "cpu_model": model, "machine": platform.machine()}


def oracle_threads(args):
    return args.cpu_threads or host_info()["nproc"]


def oracle_step_bytes(A, bs, iters):
    """Algorithmic bytes of an oracle setup + iters CG iterations (FP64 factors, same B_it)."""
    vb = 8
    setup_b = csr_bytes(A.n, A.nnz, vb) + sum(factor_bytes(A.n, bs, 8))
    _, b_it, _ = step_bytes(A.n, A.nnz, bs, "fp64", 0, vb)
    return setup_b + iters * b_it


def oracle_sample(A, b, bs, sample_iters, threads=1):
    """Oracle setup + a bounded number of CG iterations on the full matrix."""
    import oracle

    oracle.set_threads(threads)
    t0 = time.perf_counter()
    L, f = oracle.factor(A, bs)
    t1 = time.perf_counter()
    r = oracle.pcg(A, b, bs, 1e-10, max_iter=sample_iters, L=L)
    t2 = time.perf_counter()
    used = oracle.threads()
    oracle.set_threads(1)
    it = r["iterations"]
    return oracle_step_bytes(A, bs, it) / (t2 - t0) / 1e9, {"setup_s": t1 - t0, "cg_s": t2 - t1,
                                                           "iterations": it, "threads": used}


def oracle_full(A, b, bs, threads):
    """The oracle's complete FP64 setup + PCG to 1e-10 (the reference solution of the
    error-vs-oracle figures), timed on the host cores."""
    import oracle

    oracle.set_threads(threads)
    t0 = time.perf_counter()
    r = oracle.pcg(A, b, bs, 1e-10)
    s = time.perf_counter() - t0
    used = oracle.threads()
    oracle.set_threads(1)
    return r, {"seconds": s, "threads": used, "iterations": r["iterations"], "status": r["status"],
               "GBs": oracle_step_bytes(A, bs, r["iterations"]) / s / 1e9}


def rel_err(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def run_reference(args):
    rank, ws, dist = dist_init()
    if rank != 0:
        return
    A, wname, bs = single_workload(args)
    args.bs = bs
    b = W.rhs(A.n, 0)
    iters = args.cpu_sample_iters or 8
    threads = oracle_threads(args)
    vals = []
    used = 1
    for s in range(args.warmup + args.steps):
        v, meta = oracle_sample(A, b, args.bs, iters, threads)
        used = meta["threads"]
        if s >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    host = host_info()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wname, "n": A.n, "nnz": A.nnz,
                   "block_size": args.bs, "prec": "fp64"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": used, "kind": "oracle",
                         "sample": f"oracle FP64 setup + {iters} CG iterations on the full matrix per step, "
                                   f"{used} threads", "host": host},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def kappa_timing(pc, Ad, bd, bs, n, nnz, vb, steps=200):
    """Lanczos kappa before (A) and after (L^{-1} A L^{-T}) with CGS2, timed with CUDA events.
    Algorithmic bytes of step j (0-based): the operator (CSR + 2 vectors; after: + L^{-1}
    twice and 4 more vectors) plus three passes over the j+1 basis vectors (two Gram-Schmidt
    projections and the update) and the new vector."""
    import torch

    out = {}
    st = torch.cuda.current_stream()
    for name, h_bs in (("before", 0), ("after", bs)):
        H = pc.setup(Ad, h_bs, prec="fp64") if h_bs else None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        r = H.kappa(bd, max_steps=steps) if H else pc.kappa(Ad, bd, 0, max_steps=steps)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if H:
            H.destroy()
        m = r["steps"]
        op = csr_bytes(n, nnz, vb) + 16 * n
        if h_bs:
            op += 2 * factor_bytes(n, h_bs, 8)[1] + 32 * n
        byt = sum(op + 3 * (j + 1) * 8 * n + 8 * n for j in range(m))
        out[name] = {"kappa": r["kappa"], "lambda_min": r["lambda_min"], "lambda_max": r["lambda_max"],
                     "steps": m, "ms": ms, "GBs": byt / (ms / 1e3) / 1e9}
    out["note"] = "200-step Lanczos with CGS2 (FP64 factors for 'after'); bytes include the basis passes"
    return out


# ---------------------------------------------------------------- GPU helpers
def timed_solves(pc, Ad, bd, bs, prec, args, steps, warmup):
    """warmup + steps setup+solve calls (pcg_solve); returns (x, infos, ms over the timed steps)."""
    import torch

    st = torch.cuda.current_stream()
    x = info = None
    for _ in range(warmup):
        x, info = pc.pcg(Ad, bd, bs, tol=args.tol, max_iter=args.maxit, prec=prec)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(st)
    for _ in range(steps):
        x, info = pc.pcg(Ad, bd, bs, tol=args.tol, max_iter=args.maxit, prec=prec)
        infos.append(info)
    e1.record(st)
    torch.cuda.synchronize()
    return x, infos, e0.elapsed_time(e1)


def kernel_times(pc, Ad, bd, bs, prec, args):
    """Per-kernel device times of the CG loop: one extra (untimed) solve in profiling mode, where
    the loop-body kernels are launched one by one with CUDA events around each on the current
    stream.  Returns (spmv_us, precond_us, update_us, spmv_order)."""
    os.environ["PC_CG_PROFILE"] = "1"
    try:
        hp = pc.setup(Ad, bs, prec=prec)
        hp.pcg(bd, tol=args.tol, max_iter=args.maxit)
        kt = hp.trace(8)
        order = {"binned": hp.row_binned(), "col_segments": hp.col_segments(),
                 "fused_update": hp.shape()["fuse_update"] == 1}
        hp.destroy()
    finally:
        del os.environ["PC_CG_PROFILE"]
    us = [float(kt[i]) / 1e3 for i in range(3)] if len(kt) >= 3 else [0.0, 0.0, 0.0]
    return us[0], us[1], us[2], order


def kernel_table(n, nnz, vb, bs, prec, spmv_us, prec_us, upd_us, peak, peak_kind, traffic, kernel_name,
                 fused=False):
    fb = 4 if prec != "fp64" else 8
    spmv_bytes = csr_bytes(n, nnz, vb) + 2 * 8 * n                      # CSR, p (read once), q
    prec_bytes = factor_bytes(n, bs, fb)[0] + 4 * 8 * n                   # M^{-1}, r, q in; r, z out
    upd_bytes = 5 * 8 * n                                                 # x, p, z in; x, p out
    if fused:   # one kernel does both: its algorithmic bytes are the two kernels' together
        prec_bytes += upd_bytes
    gbs = lambda b, us: b / (us * 1e-6) / 1e9 if us > 0 else 0.0        # noqa: E731
    achieved = gbs(spmv_bytes, spmv_us)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel_name,
                "algorithmic_bytes_per_launch": spmv_bytes, "avg_launch_us": spmv_us}
    kernels = {
        "spmv": {"us": spmv_us, "GBs": achieved, "bytes": spmv_bytes},
        "precond": {"us": prec_us, "GBs": gbs(prec_bytes, prec_us), "bytes": prec_bytes,
                    "frac": gbs(prec_bytes, prec_us) / peak},
        "update": ({"fused_into": "precond (x += alpha p and p = z + beta p as its tail)"} if fused else
                   {"us": upd_us, "GBs": gbs(upd_bytes, upd_us), "bytes": upd_bytes,
                    "frac": gbs(upd_bytes, upd_us) / peak}),
        "note": "profiling mode: kernels launched one by one with CUDA events around each; every step "
                "starts with a 40 us spacer kernel so that the intervals exclude host launch latency",
    }
    return roofline, kernels


# ---------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch

    rank, ws, dist = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import paper_2410_02408_gb300 as pc

    pc.load()
    pc.set_row_binning(args.row_binning)
    pc.set_col_segments(args.col_segments)
    if args.ctas_per_sm:
        pc.set_ctas_per_sm(args.ctas_per_sm)
    A, wname, bs = single_workload(args)
    args.bs = bs
    vb = A.val.dtype.itemsize
    b = W.rhs(A.n, 0)
    Ad = pc.csr(A)
    bd = torch.from_numpy(b).cuda()
    n, nnz = A.n, A.nnz
    st = torch.cuda.current_stream()

    # launch shapes of the CG loop kernels, picked by the library's autotuner for each block
    # size and precision timed below (outside every timed region)
    shapes = {}

    def tuned(bsz, prec):
        if not args.no_tune and (bsz, prec) not in shapes:
            shapes[(bsz, prec)] = pc.autotune(Ad, bsz, prec, iterations=50)
        return shapes.get((bsz, prec))

    tuned(args.bs, args.prec)
    if not args.no_fp64_compare:
        tuned(args.bs, "fp64")

    for _ in range(args.warmup):
        x, info = pc.pcg(Ad, bd, args.bs, tol=args.tol, max_iter=args.maxit, prec=args.prec)
    torch.cuda.synchronize()
    barrier(dist)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(dist)
        e0.record(st)
        for _ in range(args.steps):
            x, info = pc.pcg(Ad, bd, args.bs, tol=args.tol, max_iter=args.maxit, prec=args.prec)
            infos.append(info)
        e1.record(st)
        torch.cuda.synchronize()
        barrier(dist)
    ms_total = e0.elapsed_time(e1)
    ms_total = max_over_ranks(ms_total, dist)
    ms_step = ms_total / args.steps
    iters = infos[-1]["iterations"]
    total_bytes = sum(step_bytes(n, nnz, args.bs, args.prec, inf["iterations"], vb)[0] for inf in infos)
    value = total_bytes * ws / (ms_total / 1e3) / 1e9
    solve_ms = statistics.mean(i["solve_ms"] for i in infos)
    peak, peak_kind = measured_hbm()
    _, b_it, _ = step_bytes(n, nnz, args.bs, args.prec, iters, vb)
    spmv_us, prec_us, upd_us, spmv_order = kernel_times(pc, Ad, bd, args.bs, args.prec, args)
    # the committed ncu summaries cover the 128^3 matrix at bs 16 and the 8M-row power-law matrix
    profiled = ((args.workload == "diffusion3d" and args.n == 128 and args.bs == 16)
                or (args.workload == "powerlaw_8m" and args.pl_n == 8_000_000))
    traffic = profiled_traffic(args.workload) if profiled else None
    kname = ("cg_spmv_bin_pipe_kernel (binned rows; q = A p and p.q; one launch per CG iteration)"
             if spmv_order["binned"] else "cg_spmv_kernel (q = A p and p.q; one launch per CG iteration)")
    roofline, kernels = kernel_table(n, nnz, vb, args.bs, args.prec, spmv_us, prec_us, upd_us, peak, peak_kind,
                                     traffic, kname, fused=spmv_order["fused_update"])
    # launches of this library's kernels per step: the CSR check, setup; the row-length statistic
    # (auto row order) and, when binned, the binning, cost split (3) and segment bounds; per
    # round I1, I2, arm, T; per iteration the SpMV and the preconditioner (with the update as its
    # tail) or 3 with a separate update kernel
    order_launches = (1 if args.row_binning == "auto" else 0) + (5 if spmv_order["binned"] else 0)
    per_it = 2 if spmv_order["fused_update"] else 3
    launches = sum(2 + order_launches + 4 * (i["restarts"] + 1) + per_it * i["iterations"] for i in infos)
    xr = x.cpu().numpy()
    true_res = float(np.linalg.norm(b - A.to_scipy() @ xr) / np.linalg.norm(b))   # report only

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wname, "n": n, "nnz": nnz,
                   "block_size": args.bs, "prec": "mixed (fp32 factors, fp64 CG)" if args.prec != "fp64" else "fp64",
                   "csr_values": "fp32" if vb == 4 else "fp64",
                   "tol": args.tol, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (CSR %.0f MB + factor)" % (csr_bytes(n, nnz, vb) / 1e6)},
        "iterations": iters, "true_rel_residual": true_res,
        "setup_ms": statistics.mean(i["setup_ms"] for i in infos), "solve_ms": solve_ms,
        "us_per_iteration": 1000.0 * solve_ms / max(iters, 1), "algorithmic_bytes_per_iteration": b_it,
        "frac_of_hbm_peak": value / peak,
        "roofline": roofline,
        "kernels": kernels,
        "spmv_order": spmv_order,
        "launch_shapes": {f"bs{k[0]}_{k[1]}": v for k, v in shapes.items()} or "library defaults (--no-tune)",
        "gpu_launches": launches,
    }
    line["clocks"] = clk.summary()
    x_fp64 = None

    if rank == 0 and not args.no_fp64_compare and args.prec != "fp64":
        x_fp64, finf, fms_total = timed_solves(pc, Ad, bd, args.bs, "fp64", args, 2, 1)
        fms = fms_total / 2
        fb = sum(step_bytes(n, nnz, args.bs, "fp64", fi["iterations"], vb)[0] for fi in finf) / 2
        line["fp64"] = {"value": fb / (fms / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": fms,
                        "iterations": finf[-1]["iterations"], "solve_ms": finf[-1]["solve_ms"],
                        "setup_ms": finf[-1]["setup_ms"]}
        line["mixed_speedup_vs_fp64"] = fms / ms_step

    if rank == 0 and not args.no_kappa:
        line["kappa"] = kappa_timing(pc, Ad, bd, args.bs, n, nnz, vb)

    if rank == 0 and not args.no_bs_sweep and args.workload == "diffusion3d":
        # one timed setup+solve per block size and precision (after one untimed solve)
        sweep = {}
        names = {"fp32": "mixed", "tf32": "mixed_tf32", "fp64": "fp64"}
        for bsz in (8, 16, 32, 64):
            row = {}
            for prec in ("fp32", "tf32", "fp64"):
                tuned(bsz, prec)
                _, si, sms = timed_solves(pc, Ad, bd, bsz, prec, args, 1, 1)
                si = si[-1]
                sb = step_bytes(n, nnz, bsz, prec, si["iterations"], vb)[0]
                row[names[prec]] = {
                    "ms": sms, "iterations": si["iterations"], "GBs": sb / (sms / 1e3) / 1e9,
                    "setup_ms": si["setup_ms"], "true_rel_residual": si["true_rel_residual"]}
            row["mixed_speedup_vs_fp64"] = row["fp64"]["ms"] / row["mixed"]["ms"]
            sweep[str(bsz)] = row
        line["bs_sweep"] = sweep

    if not args.no_e2e:
        line["e2e"] = e2e_single(pc, A, b, args, dist, ws)

    if rank == 0 and ws == 1:
        host = host_info()
        modes = {}
        if not args.no_cpu_baseline:
            sample = args.cpu_sample_iters or 8
            v1, m1 = oracle_sample(A, b, args.bs, sample, 1)
            modes["single"] = {"value": v1, "cores": m1["threads"],
                               "sample": f"oracle FP64 setup + {m1['iterations']} CG iterations on the full "
                                         f"matrix ({m1['setup_s'] + m1['cg_s']:.1f} s)"}
            line["cpu_baseline"] = {"value": v1, "unit": "GB/s", "cores": m1["threads"], "kind": "oracle",
                                    "sample": modes["single"]["sample"], "host": host, "modes": modes}
        if not args.no_oracle_error:
            o, om = oracle_full(A, b, args.bs, oracle_threads(args))
            modes["all_cores"] = {"value": om["GBs"], "cores": om["threads"],
                                  "sample": f"oracle FP64 setup + PCG to 1e-10 ({om['iterations']} iterations, "
                                            f"{om['seconds']:.1f} s)", "seconds_to_solution": om["seconds"]}
            if "cpu_baseline" in line:
                line["cpu_baseline"].update({"value": om["GBs"], "cores": om["threads"],
                                             "sample": modes["all_cores"]["sample"]})
            errs = {"mixed" if args.prec != "fp64" else "fp64": rel_err(xr, o["x"])}
            if x_fp64 is not None:
                errs["fp64"] = rel_err(x_fp64.cpu().numpy(), o["x"])
            errs["oracle_iterations"] = o["iterations"]
            errs["note"] = "||x - x_oracle|| / ||x_oracle||, x_oracle = the oracle's FP64 PCG to the same tolerance"
            line["err_vs_fp64_oracle"] = errs
            line["speedup_vs_oracle_all_cores"] = om["seconds"] * 1e3 / ms_step

    if rank == 0 and ws == 1 and args.workload == "diffusion3d" and not args.no_paper_rows:
        line["paper_rows"] = paper_rows(pc, A, b, Ad, bd, args)

    if rank == 0 and ws == 1 and args.workload == "diffusion3d" and not args.no_sub:
        sub = {}
        sub["batched_rgg_512"] = batched_result(pc, args, args.sub_steps, 1, tune=False)
        sub["powerlaw_8m"] = powerlaw_result(pc, args, args.sub_steps, 1)
        line["sub_workloads"] = sub
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def e2e_single(pc, A, b, args, dist, ws):
    """End to end through the C ABI from pinned host buffers: CSR and b copied in, x out."""
    import torch

    st = torch.cuda.current_stream()
    n, nnz, vb = A.n, A.nnz, A.val.dtype.itemsize
    hrp = torch.from_numpy(A.row_ptr).pin_memory()
    hci = torch.from_numpy(A.col).pin_memory()
    hva = torch.from_numpy(A.val).pin_memory()
    hb = torch.from_numpy(b).pin_memory()
    hx = torch.empty(n, dtype=torch.float64).pin_memory()
    drp = torch.empty_like(hrp, device="cuda")
    dci = torch.empty_like(hci, device="cuda")
    dva = torch.empty_like(hva, device="cuda")
    db = torch.empty_like(hb, device="cuda")
    h2d = sum(t.numel() * t.element_size() for t in (hrp, hci, hva, hb))
    d2h = hx.numel() * hx.element_size()
    torch.cuda.synchronize()
    barrier(dist)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(st)
    eb = 0
    ksteps = max(1, min(args.steps, 3))
    for _ in range(ksteps):
        drp.copy_(hrp, non_blocking=True)
        dci.copy_(hci, non_blocking=True)
        dva.copy_(hva, non_blocking=True)
        db.copy_(hb, non_blocking=True)
        xd, ei = pc.pcg(pc.CSR(drp, dci, dva), db, args.bs, tol=args.tol, max_iter=args.maxit, prec=args.prec)
        hx.copy_(xd, non_blocking=True)
        eb += step_bytes(n, nnz, args.bs, args.prec, ei["iterations"], vb)[0]
    t1.record(st)
    torch.cuda.synchronize()
    ems = max_over_ranks(t0.elapsed_time(t1), dist)
    return {"value": eb * ws / (ems / 1e3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ems / ksteps}


# ---------------------------------------------------------------- the paper's own rows
def paper_rows(pc, A, b, Ad, bd, args):
    """Point Jacobi (block size 1: the paper's preconditioner, Sec. 3.3 and its CUDA kernel in
    Sec. 4.3) setup + apply throughput against the oracle; the error of the paper's decoupled
    per-block solve x = M^-1 b (Sec. 3.2 and 3.6 solve the blocks independently) against the PCG
    solution; the paper-size sweep of kappa and kappa^2 (the HHL cost driver of Sec. 3.4) per
    block size (Sec. 5.1: N in {2^10, 2^12, 2^14})."""
    out = {}
    out["point_jacobi_bs1"] = point_jacobi_row(pc, A, b, Ad, bd, args)
    out["decoupled_solve"] = decoupled_row(pc, args)
    out["paper_size_sweep"] = paper_sweep(pc)
    out["complex_hermitian"] = complex_row(pc, args)
    return out


def complex_row(pc, args):
    """Complex Hermitian PD systems (Sec. 3.1): PCG and kappa through the real form K on the GPU,
    the error against the oracle's native complex PCG, and the oracle's time on the host cores."""
    import torch

    import oracle

    out = {}
    st = torch.cuda.current_stream()
    for wname, A, bs in (("hermitian_diffusion3d_64_sigma1", W.hermitian_diffusion3d(64, 1.0), 16),
                         ("magnetic2d_256_flux1_16", W.magnetic_laplacian_2d(256, 1.0 / 16), 16)):
        b = W.rhs_complex(A.n, 0)
        Z = pc.csr_z(A)
        bd = torch.from_numpy(b).cuda()
        pc.pcg_z(Z, bd, bs, tol=args.tol, prec="fp64")
        torch.cuda.synchronize()
        row = {"n": A.n, "nnz": A.nnz, "block_size": bs}
        for prec in ("fp64", "fp32"):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            x, info = pc.pcg_z(Z, bd, bs, tol=args.tol, prec=prec)
            e1.record(st)
            torch.cuda.synchronize()
            row[prec] = {"ms": e0.elapsed_time(e1), "iterations": info["iterations"],
                         "true_rel_residual": info["true_rel_residual"], "x": x.cpu().numpy()}
        kb = pc.kappa_z(Z, bd, 0, max_steps=200)
        ka = pc.kappa_z(Z, bd, bs, max_steps=200)
        row["kappa_before"] = kb["kappa"]
        row["kappa_after"] = ka["kappa"]
        oracle.set_threads(oracle_threads(args))
        t0 = time.perf_counter()
        o = oracle.zpcg(A, b, bs, args.tol)
        row["oracle_all_cores_s"] = time.perf_counter() - t0
        oracle.set_threads(1)
        for prec in ("fp64", "fp32"):
            row[prec]["err_vs_complex_oracle"] = rel_err(row[prec].pop("x"), o["x"])
        row["oracle_iterations"] = o["iterations"]
        out[wname] = row
    out["note"] = ("solved as the real-equivalent SPD system (2n rows, 4 nnz) with block size 2 bs; "
                   "the oracle is native complex arithmetic")
    return out


def point_jacobi_row(pc, A, b, Ad, bd, args):
    """GPU setup (CSR check + diagonal extraction + 1x1 'factor') and one application
    z = D^-1 r, against the oracle's setup + apply on the host cores, FP64 throughout.
    Bytes: setup = CSR + the two stored factor arrays; apply = factor + 2 vectors."""
    import torch

    import oracle

    st = torch.cuda.current_stream()
    n, nnz, vb = A.n, A.nnz, A.val.dtype.itemsize
    Fm, Fl = factor_bytes(n, 1, 8)
    setup_b = csr_bytes(n, nnz, vb) + Fm + Fl
    apply_b = Fm + 16 * n
    for _ in range(2):
        pc.setup(Ad, 1, prec="fp64").destroy()
    torch.cuda.synchronize()
    reps = 10
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(st)
    for _ in range(reps):
        H = pc.setup(Ad, 1, prec="fp64")
        H.destroy()
    e1.record(st)
    torch.cuda.synchronize()
    H = pc.setup(Ad, 1, prec="fp64")
    z = torch.empty_like(bd)
    H.apply("inv", bd, out=z)
    torch.cuda.synchronize()
    e1b = torch.cuda.Event(enable_timing=True)
    e1b.record(st)
    for _ in range(reps * 5):
        H.apply("inv", bd, out=z)
    e2.record(st)
    torch.cuda.synchronize()
    setup_ms = e0.elapsed_time(e1) / reps
    apply_ms = e1b.elapsed_time(e2) / (reps * 5)
    zr = z.cpu().numpy()
    H.destroy()
    row = {"gpu": {"setup_ms": setup_ms, "apply_ms": apply_ms,
                   "setup_GBs": setup_b / (setup_ms / 1e3) / 1e9, "apply_GBs": apply_b / (apply_ms / 1e3) / 1e9,
                   "note": "setup = pc_setup + pc_destroy (CSR check, extraction, factor allocation and writes)"}}
    for mode, threads in (("single", 1), ("all_cores", oracle_threads(args))):
        oracle.set_threads(threads)
        t0 = time.perf_counter()
        L, _ = oracle.factor(A, 1)
        t1 = time.perf_counter()
        k = 3
        for _ in range(k):
            zo = oracle.apply(A, L, 1, oracle.MODE_INV, b)
        t2 = time.perf_counter()
        row[mode] = {"setup_ms": (t1 - t0) * 1e3, "apply_ms": (t2 - t1) * 1e3 / k, "cores": oracle.threads()}
        oracle.set_threads(1)
    row["max_abs_diff_vs_oracle"] = float(np.max(np.abs(zr - zo)))
    for mode in ("single", "all_cores"):
        row[f"speedup_vs_{mode}"] = {"setup": row[mode]["setup_ms"] / setup_ms,
                                     "apply": row[mode]["apply_ms"] / apply_ms,
                                     "setup_plus_apply": (row[mode]["setup_ms"] + row[mode]["apply_ms"]) /
                                                         (setup_ms + apply_ms)}
    row["workload"] = "diffusion3d 128^3 sigma 2 (the headline matrix), FP64"
    row["paper"] = "Sec. 5.3.1 reports up to 15x for its CUDA point-Jacobi preconditioning over CPU (GPU, CPU unstated)"
    return row


def decoupled_row(pc, args):
    """x_dec = M^-1 b (each block solved on its own, the solution the paper assembles from the
    blocks) against the PCG solution x of the full system: ||x_dec - x|| / ||x|| and the
    residual ||b - A x_dec|| / ||b||, per block size, FP64 factors."""
    import torch

    out = {}
    for wname, A in (("poisson2d_64", W.poisson2d(64)), ("diffusion3d_128_sigma2", W.diffusion3d(128, 2.0))):
        b = W.rhs(A.n, 0)
        Ad = pc.csr(A)
        bd = torch.from_numpy(b).cuda()
        Asp = A.to_scipy()
        rows = {}
        for bs in (1, 8, 16, 32, 64):
            H = pc.setup(Ad, bs, prec="fp64")
            try:
                xd = H.apply("inv", bd).cpu().numpy()
                x, info = H.pcg(bd, tol=args.tol, max_iter=args.maxit)
            finally:
                H.destroy()
            x = x.cpu().numpy()
            rows[str(bs)] = {"err_vs_pcg": rel_err(xd, x),
                             "rel_residual": float(np.linalg.norm(b - Asp @ xd) / np.linalg.norm(b)),
                             "pcg_iterations": info["iterations"]}
        out[wname] = rows
    return out


def paper_sweep(pc):
    """kappa before and after block-Jacobi preconditioning and the kappa^2 reduction (HHL's cost
    grows as kappa^2, Sec. 3.4) at the paper's sizes N = 2^10, 2^12, 2^14 (Sec. 5.1): 2D Poisson
    and random SPD matrices of three densities (power-law recipe, mean off-diagonal degree 4,
    8, 16).  Lanczos with min(N, 200) steps and CGS2; PCG iterations to 1e-10 per block size."""
    import torch

    out = {}
    for N in (1024, 4096, 16384):
        mats = [(f"poisson2d_{int(round(N ** 0.5))}", W.poisson2d(int(round(N ** 0.5))))]
        for d in (4, 8, 16):
            mats.append((f"random_spd_deg{d}", W.random_spd(N, d)))
        res = {}
        for name, A in mats:
            b = W.rhs(A.n, 0)
            Ad = pc.csr(A)
            bd = torch.from_numpy(b).cuda()
            m = min(A.n, 200)
            kb = pc.kappa(Ad, bd, 0, max_steps=m)
            row = {"nnz": A.nnz, "kappa_before": kb["kappa"], "steps": kb["steps"], "by_bs": {}}
            for bs in (1, 4, 16, 64):
                H = pc.setup(Ad, bs, prec="fp64")
                try:
                    ka = H.kappa(bd, max_steps=m)
                    _, info = H.pcg(bd, tol=1e-10)
                finally:
                    H.destroy()
                row["by_bs"][str(bs)] = {"kappa_after": ka["kappa"],
                                         "kappa2_reduction": (kb["kappa"] / ka["kappa"]) ** 2,
                                         "pcg_iterations": info["iterations"]}
            res[name] = row
        out[str(N)] = res
    return out


# ---------------------------------------------------------------- batched workload
def batch_step_bytes(batch, prec, iters, restarts):
    """Algorithmic bytes of one batched step: per system, setup (CSR read, M^{-1} write),
    the x0 = 0 start (b read, M^{-1} read, x, r, z, p written), iterations * B_it and the
    true residual (CSR, x, b read, r written), plus one M^{-1} pass and 5 vectors per restart."""
    fb = 4 if prec != "fp64" else 8
    total = 0
    for s, A in enumerate(batch.systems):
        n, nnz, bs = A.n, A.nnz, int(batch.bs[s])
        C = csr_bytes(n, nnz, 8)
        Fm, _ = factor_bytes(n, bs, fb)
        v = 8 * n
        b_it = C + Fm + 11 * v
        total += (C + Fm) + (Fm + 5 * v) + int(iters[s]) * b_it + (int(restarts[s]) + 1) * (C + 3 * v)
        total += int(restarts[s]) * (Fm + 5 * v)
    return total


def batched_result(pc, args, steps, warmup, tune=True):
    """Setup + PCG of the 512 uneven RGG systems in one persistent launch: the figures of one
    JSON line (returned as a dict)."""
    import torch

    t0 = time.time()
    batch = W.rgg_batch(n_sys=args.n_sys, seed=3)
    gen_s = time.time() - t0
    n_rows = int(batch.sys_row[-1])
    nnz = int(batch.row_ptr[-1])
    b = W.rhs(n_rows, 0)
    bd = torch.from_numpy(b).cuda()
    st = torch.cuda.current_stream()
    peak, peak_kind = measured_hbm()
    tuning = {}
    use_defaults = not args.batch_shape and not (tune and not args.no_tune)

    def set_shape(sh):
        occ, team, split, kb = sh.split(",")
        pc.batch_set_tuning(int(occ), int(team), float(split))
        pc.binding.lib().pc_batch_set_setup_smem(int(kb))

    if args.batch_shape:
        set_shape(args.batch_shape)
        tuning["explicit"] = args.batch_shape
    elif use_defaults:
        tuning["explicit"] = dict(BATCH_SHAPE_DEFAULT)
    else:
        for prec in ([args.prec, "fp64"] if args.prec != "fp64" and not args.no_fp64_compare else [args.prec]):
            t0 = time.time()
            tms, cfg = pc.batch_autotune(batch, bd, args.tol, args.maxit, prec, args.tune_trials)
            tuning[prec] = {"best_ms": tms, "config": cfg, "tuning_s": time.time() - t0}

    def timed(prec, nsteps, nwarm):
        if use_defaults:
            set_shape(BATCH_SHAPE_DEFAULT.get(prec, BATCH_SHAPE_DEFAULT["fp32"]))
        H = pc.Batch(batch, prec)
        x = torch.empty_like(bd)
        for _ in range(nwarm):
            H.solve(bd, args.tol, args.maxit, x=x)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        per = info = None
        kms = []
        e0.record(st)
        for _ in range(nsteps):
            _, per, info = H.solve(bd, args.tol, args.maxit, x=x)
            kms.append(info["solve_ms"])
        e1.record(st)
        torch.cuda.synchronize()
        li = H.launch_info()
        team, _ = H.teams()
        H.destroy()
        ms = e0.elapsed_time(e1) / nsteps
        return x, per, info, ms, statistics.mean(kms), li, team

    with ClockSampler(0) as clk:
        x, per, info, ms, kms, li, team = timed(args.prec, steps, warmup)
    restarts = np.zeros(batch.n_sys, dtype=np.int64)   # per-system restarts are not exported; bytes omit them
    step_b = batch_step_bytes(batch, args.prec, per["iterations"], restarts)
    value = step_b / (ms / 1e3) / 1e9
    achieved = step_b / (kms / 1e3) / 1e9
    it = per["iterations"]
    res = {
        "metric": METRIC, "value": value, "unit": "GB/s", "ms_per_step": ms, "steps": steps, "warmup": warmup,
        "config": {"workload": f"batched_rgg_{batch.n_sys}", "n_sys": batch.n_sys, "rows": n_rows, "nnz": nnz,
                   "block_sizes": "per system from {4,8,16,32,64}",
                   "prec": "mixed (fp32 factors, fp64 CG)" if args.prec != "fp64" else "fp64", "tol": args.tol,
                   "parallelism": "one persistent launch, teams of CTAs per system",
                   "l2": "inputs larger than L2 (CSR %.0f MB)" % (csr_bytes(n_rows, nnz, 8) / 1e6)},
        "status": info["status_name"], "worst_true_rel_residual": float(np.max(per["relres"])),
        "iterations": {"min": int(it.min()), "median": float(np.median(it)), "max": int(it.max()),
                       "sum": int(it.sum())},
        "frac_of_hbm_peak": value / peak,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_kind": peak_kind,
                     "kernel": "batched_kernel (setup + PCG of every system, one persistent launch)",
                     "algorithmic_bytes_per_launch": step_b, "avg_launch_us": kms * 1e3},
        "launch": li, "teams": {"multi_cta_systems": int((team > 1).sum()), "max_team": int(team.max())},
        "graph": bool(info["graph"]), "gpu_launches": 2 * steps, "generation_s": gen_s, "autotune": tuning,
    }
    res["clocks"] = clk.summary()
    x_mixed = x.cpu().numpy()
    if args.phase_profile:
        os.environ["PC_BATCH_PROFILE"] = "1"
        Hp = pc.Batch(batch, args.prec)
        Hp.solve(bd, args.tol, args.maxit)
        prof = Hp.phase_profile()
        Hp.destroy()
        del os.environ["PC_BATCH_PROFILE"]
        tot = sum(prof.values()) or 1
        res["phase_profile"] = {k: {"cta_ms": v / 1e6, "share": v / tot} for k, v in prof.items()}
    x64 = None
    if args.prec != "fp64" and not args.no_fp64_compare:
        x64t, per64, info64, ms64, kms64, _, _ = timed("fp64", max(1, min(steps, 2)), 1)
        x64 = x64t.cpu().numpy()
        b64 = batch_step_bytes(batch, "fp64", per64["iterations"], restarts)
        res["fp64"] = {"value": b64 / (ms64 / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": ms64,
                       "iterations_sum": int(per64["iterations"].sum()), "status": info64["status_name"]}
        res["mixed_speedup_vs_fp64"] = ms64 / ms
    if not args.no_e2e:
        hb = torch.from_numpy(b).pin_memory()
        hx = torch.empty(n_rows, dtype=torch.float64).pin_memory()
        hrp = torch.from_numpy(batch.row_ptr).pin_memory()
        hci = torch.from_numpy(batch.col).pin_memory()
        hva = torch.from_numpy(batch.val).pin_memory()
        if use_defaults:
            set_shape(BATCH_SHAPE_DEFAULT.get(args.prec, BATCH_SHAPE_DEFAULT["fp32"]))
        H = pc.Batch(batch, args.prec)
        dbb = torch.empty_like(hb, device="cuda")
        xe = torch.empty_like(dbb)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        k = max(1, min(steps, 3))
        for _ in range(k):
            H.row_ptr.copy_(hrp, non_blocking=True)
            H.col.copy_(hci, non_blocking=True)
            H.val.copy_(hva, non_blocking=True)
            dbb.copy_(hb, non_blocking=True)
            H.solve(dbb, args.tol, args.maxit, x=xe)
            hx.copy_(xe, non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        H.destroy()
        ems = e0.elapsed_time(e1) / k
        h2d = sum(t.numel() * t.element_size() for t in (hrp, hci, hva, hb))
        res["e2e"] = {"value": step_b / (ems / 1e3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": hx.numel() * 8, "ms_per_step": ems}
    if not args.no_cpu_baseline or not args.no_oracle_error:
        import oracle

        # oracle PCG of sampled systems (smallest, median and largest sizes) on all host cores:
        # the error of each result against it, and the oracle's throughput on that sample
        threads = oracle_threads(args)
        oracle.set_threads(threads)
        sizes = np.array([A.n for A in batch.systems])
        order = np.argsort(sizes)
        sample = list(order[:4]) + list(order[len(order) // 2 - 2:len(order) // 2 + 2]) + list(order[-2:])
        errs_m, errs_64 = [], []
        sb = 0
        t0 = time.perf_counter()
        for s in sample:
            A = batch.systems[s]
            sl = slice(int(batch.sys_row[s]), int(batch.sys_row[s + 1]))
            r = oracle.pcg(A, b[sl], int(batch.bs[s]), args.tol)
            errs_m.append(rel_err(x_mixed[sl], r["x"]))
            if x64 is not None:
                errs_64.append(rel_err(x64[sl], r["x"]))
            n_s, nnz_s, bs_s = A.n, A.nnz, int(batch.bs[s])
            C = csr_bytes(n_s, nnz_s, 8)
            Fm, _ = factor_bytes(n_s, bs_s, 8)
            v = 8 * n_s
            sb += (C + Fm) + (Fm + 5 * v) + r["iterations"] * (C + Fm + 11 * v) + (r["restarts"] + 1) * (C + 3 * v)
        cs = time.perf_counter() - t0
        used = oracle.threads()
        oracle.set_threads(1)
        res["err_vs_fp64_oracle"] = {"mixed_max": max(errs_m), "fp64_max": max(errs_64) if errs_64 else None,
                                     "systems": [int(s) for s in sample],
                                     "note": "max over sampled systems of ||x_s - x_oracle,s|| / ||x_oracle,s||"}
        res["cpu_baseline"] = {"value": sb / cs / 1e9, "unit": "GB/s", "cores": used, "kind": "oracle",
                               "sample": f"oracle FP64 setup + PCG of {len(sample)} sampled systems ({cs:.1f} s)"}
    return res


def run_batched(args):
    import paper_2410_02408_gb300 as pc

    pc.load()
    res = batched_result(pc, args, args.steps, args.warmup, tune=True)
    line = {"n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic"}
    line.update(res)
    print(json.dumps(line))


# ---------------------------------------------------------------- power-law workload
def powerlaw_result(pc, args, steps, warmup):
    """The 8M-row power-law matrix (FP32 values, bs 32): mixed and FP64-factor setup + solve,
    the binned SpMV's roofline, and the error against the oracle's FP64 PCG."""
    import torch

    t0 = time.time()
    A = W.powerlaw_spd(args.pl_n, seed=5)
    gen_s = time.time() - t0
    bs = 32
    b = W.rhs(A.n, 0)
    Ad = pc.csr(A)
    bd = torch.from_numpy(b).cuda()
    n, nnz, vb = A.n, A.nnz, A.val.dtype.itemsize
    peak, peak_kind = measured_hbm()
    # launch shapes of the loop kernels (binned row loop, ring depth) from the autotuner
    shapes = {} if args.no_tune else {p: pc.autotune(Ad, bs, p, iterations=30) for p in (args.prec, "fp64")}
    with ClockSampler(0) as clk:
        x, infos, ms_total = timed_solves(pc, Ad, bd, bs, args.prec, args, steps, warmup)
    ms = ms_total / steps
    byt = sum(step_bytes(n, nnz, bs, args.prec, i["iterations"], vb)[0] for i in infos)
    value = byt / (ms_total / 1e3) / 1e9
    spmv_us, prec_us, upd_us, order = kernel_times(pc, Ad, bd, bs, args.prec, args)
    kname = ("cg_spmv_bin_pipe_kernel (binned rows; q = A p and p.q; one launch per CG iteration)"
             if order["binned"] else "cg_spmv_kernel (q = A p and p.q; one launch per CG iteration)")
    traffic = profiled_traffic("powerlaw_8m") if n == 8_000_000 and args.prec != "fp64" else None
    roofline, kernels = kernel_table(n, nnz, vb, bs, args.prec, spmv_us, prec_us, upd_us, peak, peak_kind, traffic,
                                     kname, fused=order["fused_update"])
    info = infos[-1]
    res = {"metric": METRIC, "value": value, "unit": "GB/s", "ms_per_step": ms, "steps": steps, "warmup": warmup,
           "config": {"workload": f"powerlaw_{n}_fp32vals", "n": n, "nnz": nnz, "block_size": bs,
                      "prec": "mixed (fp32 factors, fp64 CG)" if args.prec != "fp64" else "fp64",
                      "csr_values": "fp32" if vb == 4 else "fp64", "tol": args.tol,
                      "l2": "inputs larger than L2 (CSR %.0f MB + factor)" % (csr_bytes(n, nnz, vb) / 1e6)},
           "iterations": info["iterations"], "true_rel_residual": info["true_rel_residual"],
           "setup_ms": statistics.mean(i["setup_ms"] for i in infos),
           "solve_ms": statistics.mean(i["solve_ms"] for i in infos),
           "frac_of_hbm_peak": value / peak, "roofline": roofline, "kernels": kernels, "spmv_order": order,
           "launch_shapes": shapes or "library defaults (--no-tune)",
           "generation_s": gen_s,
           "gpu_launches": sum(2 + 6 + 4 * (i["restarts"] + 1) + (2 if order["fused_update"] else 3) * i["iterations"]
                               for i in infos)}
    res["clocks"] = clk.summary()
    x64 = None
    if args.prec != "fp64" and not args.no_fp64_compare:
        x64t, finf, fms_total = timed_solves(pc, Ad, bd, bs, "fp64", args, 1, 1)
        x64 = x64t.cpu().numpy()
        fb = step_bytes(n, nnz, bs, "fp64", finf[-1]["iterations"], vb)[0]
        res["fp64"] = {"value": fb / (fms_total / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": fms_total,
                       "iterations": finf[-1]["iterations"]}
        res["mixed_speedup_vs_fp64"] = fms_total / ms
    if not args.no_oracle_error:
        o, om = oracle_full(A, b, bs, oracle_threads(args))
        errs = {"mixed" if args.prec != "fp64" else "fp64": rel_err(x.cpu().numpy(), o["x"])}
        if x64 is not None:
            errs["fp64"] = rel_err(x64, o["x"])
        errs["oracle_iterations"] = o["iterations"]
        res["err_vs_fp64_oracle"] = errs
        res["cpu_baseline"] = {"value": om["GBs"], "unit": "GB/s", "cores": om["threads"], "kind": "oracle",
                               "sample": f"oracle FP64 setup + PCG to 1e-10 ({om['iterations']} iterations, "
                                         f"{om['seconds']:.1f} s)", "seconds_to_solution": om["seconds"]}
    return res


def main():
    args = parse()
    if args.profile:
        run_profile(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched_rgg_512":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
