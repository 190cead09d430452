"""Benchmark: block-Jacobi PCG to relative residual 1e-10 on the 3D variable-coefficient
diffusion workload (128^3 grid, 7-point stencil, log-normal face coefficients with
sigma = 2, b ~ N(0,1) seed 0), mixed precision (FP32 block factors, FP64 CG) against
all-FP64.

One step = pcg_solve through the C ABI: block extraction + batched block Cholesky/inverse
(setup) and the CG solve (a CUDA graph with a device-driven loop) to ||r||/||b|| <= 1e-10
with the true-residual check.  The line also carries the per-kernel breakdown, the roofline
of the dominant kernel (the SpMV), the FP64-factor comparison, the Lanczos kappa estimates
before and after preconditioning, the end-to-end figure and the oracle's CPU baseline.

Other workloads (each prints its own line): --workload batched_rgg_512 (512 uneven RGG
systems set up and solved in one persistent launch) and --workload powerlaw_8m (random SPD
with power-law rows, FP32 values).

value   = algorithmic bytes of the step / step time (GB/s), inputs resident in HBM.
          bytes = setup (CSR read + factor writes) + per-solve extras (initial and final
          residual, final x update) + iterations * B_it, where
          B_it = CSR (val+col+row_ptr) + M^{-1} factor + 11 vector streams of 8N bytes.
e2e     = the same metric through the C ABI with host buffers: the CSR and b are copied
          from pinned host memory to the device and x back inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
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


def parse():
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
    ap.add_argument("--cpu-sample-iters", type=int, default=0, help="oracle CG iterations per sample (0 = auto)")
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
    ap.add_argument("--no-tune", action="store_true", help="batched workload: skip the launch-shape autotuner")
    ap.add_argument("--tune-trials", type=int, default=0, help="batched autotuner candidates (0 = all)")
    ap.add_argument("--batch-shape", default="",
                    help="batched workload: explicit launch shape 'ctas_per_sm,team_max,slots_per_cta,setup_kb' "
                         "(skips the autotuner)")
    ap.add_argument("--phase-profile", action="store_true",
                    help="batched workload: one extra solve with per-phase device timers (not timed)")
    ap.add_argument("--profile", action="store_true",
                    help="one solve of the workload and nothing else (for ncu captures); prints a short line")
    args = ap.parse_args()
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


# Sources that define the profiled CG SpMV kernel: its recorded DRAM traffic stays valid
# while these files are unchanged.
SPMV_SOURCES = ("pc_cg_graph.cu", "pc_common.cuh", "pc_kernels.cuh", "pc_tma.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2410_02408_gb300", "csrc")
    for fn in SPMV_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(bs, prec):
    """DRAM bytes per launch of the SpMV kernel from the committed ncu summary, or None if
    absent or if the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "cg_spmv_kernel_diffusion3d_128.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_hash:\s*(\w+)", txt)
    if not m or m.group(1) != kernel_source_hash():
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
def oracle_sample(A, b, bs, sample_iters):
    """Oracle setup + a bounded number of CG iterations on the full matrix (single thread)."""
    import oracle

    t0 = time.perf_counter()
    L, f = oracle.factor(A, bs)
    t1 = time.perf_counter()
    r = oracle.pcg(A, b, bs, 1e-10, max_iter=sample_iters, L=L)
    t2 = time.perf_counter()
    it = r["iterations"]
    setup_b = csr_bytes(A.n, A.nnz, 8) + factor_bytes(A.n, bs, 8)[0] + factor_bytes(A.n, bs, 8)[1]
    _, b_it, _ = step_bytes(A.n, A.nnz, bs, "fp64", 0)
    byt = setup_b + it * b_it
    return byt / (t2 - t0) / 1e9, {"setup_s": t1 - t0, "cg_s": t2 - t1, "iterations": it}


def run_reference(args):
    rank, ws, dist = dist_init()
    if rank != 0:
        return
    A, wname, bs = single_workload(args)
    args.bs = bs
    b = W.rhs(A.n, 0)
    iters = args.cpu_sample_iters or 8
    vals = []
    for s in range(args.warmup + args.steps):
        v, meta = oracle_sample(A, b, args.bs, iters)
        if s >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wname, "n": A.n, "nnz": A.nnz,
                   "block_size": args.bs, "prec": "fp64"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"oracle setup + {iters} CG iterations on the full matrix per step"},
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

    def solve(prec):
        x, info = pc.pcg(Ad, bd, args.bs, tol=args.tol, max_iter=args.maxit, prec=prec)
        return x, info

    for _ in range(args.warmup):
        x, info = solve(args.prec)
    torch.cuda.synchronize()
    barrier(dist)
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(dist)
        e0.record(st)
        for _ in range(args.steps):
            x, info = solve(args.prec)
            infos.append(info)
        e1.record(st)
        torch.cuda.synchronize()
        barrier(dist)
    ms_total = e0.elapsed_time(e1)
    ms_total = max_over_ranks(ms_total, dist)
    ms_step = ms_total / args.steps
    iters = infos[-1]["iterations"]
    total_bytes = 0
    for inf in infos:
        sb, b_it, kb = step_bytes(n, nnz, args.bs, args.prec, inf["iterations"], vb)
        total_bytes += sb
    value = total_bytes * ws / (ms_total / 1e3) / 1e9
    solve_ms = statistics.mean(i["solve_ms"] for i in infos)
    peak, peak_kind = measured_hbm()
    _, b_it, _ = step_bytes(n, nnz, args.bs, args.prec, iters, vb)
    # Per-kernel times: one extra (untimed) solve in profiling mode, where the loop-body
    # kernels are launched one by one with CUDA events around each on the current stream.
    os.environ["PC_CG_PROFILE"] = "1"
    hp = pc.setup(Ad, args.bs, prec=args.prec)
    hp.pcg(bd, tol=args.tol, max_iter=args.maxit)
    kt = hp.trace(8)
    spmv_order = {"binned": hp.row_binned(), "col_segments": hp.col_segments()}
    hp.destroy()
    del os.environ["PC_CG_PROFILE"]
    spmv_us, prec_us, upd_us = (float(kt[0]) / 1e3, float(kt[1]) / 1e3, float(kt[2]) / 1e3) if len(kt) >= 3 else (0.0, 0.0, 0.0)
    fb = 4 if args.prec != "fp64" else 8
    spmv_bytes = csr_bytes(n, nnz, vb) + 2 * 8 * n                      # CSR, p (read once), q
    prec_bytes = factor_bytes(n, args.bs, fb)[0] + 4 * 8 * n              # M^{-1}, r, q in; r, z out
    upd_bytes = 5 * 8 * n                                                 # x, p, z in; x, p out
    # dominant kernel (largest share of the iteration): the SpMV q = A p with the p.q reduction
    achieved = spmv_bytes / (spmv_us * 1e-6) / 1e9 if spmv_us > 0 else 0.0
    traffic = profiled_traffic(args.bs, args.prec) if args.workload == "diffusion3d" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "cg_spmv_kernel (q = A p and p.q; one launch per CG iteration)",
                "algorithmic_bytes_per_launch": spmv_bytes, "avg_launch_us": spmv_us}
    kernels = {
        "spmv": {"us": spmv_us, "GBs": achieved, "bytes": spmv_bytes},
        "precond": {"us": prec_us, "GBs": prec_bytes / (prec_us * 1e-6) / 1e9 if prec_us > 0 else 0.0,
                    "bytes": prec_bytes},
        "update": {"us": upd_us, "GBs": upd_bytes / (upd_us * 1e-6) / 1e9 if upd_us > 0 else 0.0,
                   "bytes": upd_bytes},
        "note": "profiling-mode launches (events around each kernel), includes per-launch overhead",
    }
    # launches of this library's kernels per step: setup; the row-length statistic (auto row
    # order) and, when binned, the binning, cost split (3) and segment bounds; per round I1,
    # I2, arm, T; 3 per iteration
    order_launches = (1 if args.row_binning == "auto" else 0) + (5 if spmv_order["binned"] else 0)
    launches = sum(1 + order_launches + 4 * (i["restarts"] + 1) + 3 * i["iterations"] for i in infos)
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
        "gpu_launches": launches,
    }
    line["clocks"] = clk.summary()

    if rank == 0 and not args.no_fp64_compare and args.prec != "fp64":
        torch.cuda.synchronize()
        solve("fp64")
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(st)
        reps = 2
        finf = []
        for _ in range(reps):
            _, fi = solve("fp64")
            finf.append(fi)
        t1.record(st)
        torch.cuda.synchronize()
        fms = t0.elapsed_time(t1) / reps
        fb = sum(step_bytes(n, nnz, args.bs, "fp64", fi["iterations"], vb)[0] for fi in finf) / reps
        line["fp64"] = {"value": fb / (fms / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": fms,
                        "iterations": finf[-1]["iterations"], "solve_ms": finf[-1]["solve_ms"],
                        "setup_ms": finf[-1]["setup_ms"]}
        line["mixed_speedup_vs_fp64"] = fms / ms_step

    if rank == 0 and not args.no_kappa:
        line["kappa"] = kappa_timing(pc, Ad, bd, args.bs, n, nnz, vb)

    if rank == 0 and not args.no_bs_sweep and args.workload == "diffusion3d":
        # one timed setup+solve per block size and precision (after one untimed solve)
        sweep = {}
        for bsz in (8, 16, 32, 64):
            row = {}
            for prec in ("fp32", "fp64"):
                pc.pcg(Ad, bd, bsz, tol=args.tol, max_iter=args.maxit, prec=prec)
                torch.cuda.synchronize()
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record(st)
                _, si = pc.pcg(Ad, bd, bsz, tol=args.tol, max_iter=args.maxit, prec=prec)
                t1.record(st)
                torch.cuda.synchronize()
                sms = t0.elapsed_time(t1)
                sb = step_bytes(n, nnz, bsz, prec, si["iterations"], vb)[0]
                row["mixed" if prec == "fp32" else "fp64"] = {
                    "ms": sms, "iterations": si["iterations"], "GBs": sb / (sms / 1e3) / 1e9,
                    "true_rel_residual": si["true_rel_residual"]}
            row["mixed_speedup_vs_fp64"] = row["fp64"]["ms"] / row["mixed"]["ms"]
            sweep[str(bsz)] = row
        line["bs_sweep"] = sweep

    if not args.no_e2e:
        # end to end through the C ABI from pinned host buffers
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
        line["e2e"] = {"value": eb * ws / (ems / 1e3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": ems / ksteps}

    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        sample = args.cpu_sample_iters or 8
        v, meta = oracle_sample(A, b, args.bs, sample)
        line["cpu_baseline"] = {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                "sample": f"oracle FP64 setup + {meta['iterations']} CG iterations on the full "
                                          f"matrix ({meta['setup_s'] + meta['cg_s']:.1f} s)"}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


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


def run_batched(args):
    import torch

    import paper_2410_02408_gb300 as pc

    pc.load()
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
    if args.batch_shape:
        occ, team, split, kb = args.batch_shape.split(",")
        pc.batch_set_tuning(int(occ), int(team), float(split))
        pc.binding.lib().pc_batch_set_setup_smem(int(kb))
        tuning["explicit"] = args.batch_shape
    elif not args.no_tune:
        for prec in ([args.prec, "fp64"] if args.prec != "fp64" and not args.no_fp64_compare else [args.prec]):
            t0 = time.time()
            tms, cfg = pc.batch_autotune(batch, bd, args.tol, args.maxit, prec, args.tune_trials)
            tuning[prec] = {"best_ms": tms, "config": cfg, "tuning_s": time.time() - t0}

    def timed(prec, steps, warmup):
        H = pc.Batch(batch, prec)
        x = torch.empty_like(bd)
        for _ in range(warmup):
            H.solve(bd, args.tol, args.maxit, x=x)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        per = info = None
        kms = []
        e0.record(st)
        for _ in range(steps):
            _, per, info = H.solve(bd, args.tol, args.maxit, x=x)
            kms.append(info["solve_ms"])
        e1.record(st)
        torch.cuda.synchronize()
        li = H.launch_info()
        team, _ = H.teams()
        H.destroy()
        ms = e0.elapsed_time(e1) / steps
        return x, per, info, ms, statistics.mean(kms), li, team

    with ClockSampler(0) as clk:
        x, per, info, ms, kms, li, team = timed(args.prec, args.steps, args.warmup)
    restarts = np.zeros(batch.n_sys, dtype=np.int64)   # per-system restarts are not exported; bytes omit them
    step_b = batch_step_bytes(batch, args.prec, per["iterations"], restarts)
    value = step_b / (ms / 1e3) / 1e9
    achieved = step_b / (kms / 1e3) / 1e9
    it = per["iterations"]
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
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
        "graph": bool(info["graph"]), "gpu_launches": 2 * args.steps, "generation_s": gen_s, "autotune": tuning,
    }
    line["clocks"] = clk.summary()
    if args.phase_profile:
        os.environ["PC_BATCH_PROFILE"] = "1"
        Hp = pc.Batch(batch, args.prec)
        Hp.solve(bd, args.tol, args.maxit)
        prof = Hp.phase_profile()
        Hp.destroy()
        del os.environ["PC_BATCH_PROFILE"]
        tot = sum(prof.values()) or 1
        line["phase_profile"] = {k: {"cta_ms": v / 1e6, "share": v / tot} for k, v in prof.items()}
    if args.prec != "fp64" and not args.no_fp64_compare:
        _, per64, info64, ms64, kms64, _, _ = timed("fp64", max(1, min(args.steps, 2)), 1)
        b64 = batch_step_bytes(batch, "fp64", per64["iterations"], restarts)
        line["fp64"] = {"value": b64 / (ms64 / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": ms64,
                        "iterations_sum": int(per64["iterations"].sum()), "status": info64["status_name"]}
        line["mixed_speedup_vs_fp64"] = ms64 / ms
    if not args.no_e2e:
        hb = torch.from_numpy(b).pin_memory()
        hx = torch.empty(n_rows, dtype=torch.float64).pin_memory()
        hrp = torch.from_numpy(batch.row_ptr).pin_memory()
        hci = torch.from_numpy(batch.col).pin_memory()
        hva = torch.from_numpy(batch.val).pin_memory()
        H = pc.Batch(batch, args.prec)
        dbb = torch.empty_like(hb, device="cuda")
        xe = torch.empty_like(dbb)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        k = max(1, min(args.steps, 3))
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
        line["e2e"] = {"value": step_b / (ems / 1e3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": hx.numel() * 8, "ms_per_step": ems}
    if not args.no_cpu_baseline:
        import oracle

        # systems in increasing size until about 10 s of CPU work
        order = np.argsort([A.n for A in batch.systems])
        t0 = time.perf_counter()
        sb = 0
        done = 0
        for s in order:
            if time.perf_counter() - t0 > 10.0:
                break
            done += 1
            A = batch.systems[s]
            sl = slice(int(batch.sys_row[s]), int(batch.sys_row[s + 1]))
            r = oracle.pcg(A, b[sl], int(batch.bs[s]), args.tol)
            n_s, nnz_s, bs_s = A.n, A.nnz, int(batch.bs[s])
            C = csr_bytes(n_s, nnz_s, 8)
            Fm, _ = factor_bytes(n_s, bs_s, 8)
            v = 8 * n_s
            sb += (C + Fm) + (Fm + 5 * v) + r["iterations"] * (C + Fm + 11 * v) + (r["restarts"] + 1) * (C + 3 * v)
        cs = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sb / cs / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                "sample": f"oracle FP64 setup + PCG of the {done} smallest systems ({cs:.1f} s)"}
    print(json.dumps(line))


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
