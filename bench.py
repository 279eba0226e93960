#!/usr/bin/env python3
"""Benchmark: time-to-solution of the asynchronous cascaded CG solve.

Workload (one "step"): CG to relative residual 1e-10 in FP64 on the 3D 7-point
Poisson matrix of a 128^3 grid (n = 2,097,152, nnz = 14,581,760), b = A x*
with x* ~ U[-1, 1] (seed 2002), x0 = 0.  The solve starts at once on the
default CSR-scalar kernel while the side stream extracts the Table IV
features, runs the cascade (FORMAT -> ALGO -> PARAM) and converts the format;
the solve switches kernel mid-run (Sec. III-C).  Each step starts from the
freshly loaded CSR (converted formats and features dropped), so the
preprocessing is inside every measured time-to-solution.

Printed JSON line: value = mean time-to-solution (ms, CUDA events around each
solve on the main stream); plus the plain CSR-scalar CG and the sequential
(predict-then-solve) and FP32-inner refinement variants, the SpMV roofline,
the CPU oracle baseline, the end-to-end time through host buffers, clocks and
kernel counts, and a GMRES(30) leg on convection-diffusion 96^3 (asynchronous
cascade, FP32 inner solves, per-step launches, the persistent kernel's FP64
FMA rate).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "time-to-solution (incl. prep) vs plain CSR-CG; SpMV % HBM BW; serve p50/p99"
GRID = 128
TOL = 1e-10
XSTAR_SEED = 2002
# FP32 refinement: each inner solve to relative max(1e-5, IR_THETA tol ||b|| / ||r||)
IR_THETA = 0.5


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_init(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=10.0):
        """Block until the first sample arrives: nvidia-smi's start-up (driver
        queries that can briefly hold up CUDA calls) then falls outside the
        timed region."""
        t0 = time.time()
        while self.proc and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.02)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload():
    from paper_2411_10143_b300 import workloads as W
    A = W.poisson3d(GRID)
    xs = W.vector(A.nrows, XSTAR_SEED)
    return A, xs


def spmv_bytes(A):
    """Algorithmic bytes of one FP64 SpMV with int32 indices, one definition for
    every configuration: the CSR matrix (val, col, rowptr), x read once and y
    written once, 12 nnz + 4 (n+1) + 8 ncols + 8 n.  Padding and repeated x
    gathers are not counted, so every format is measured against the same
    work and the fractions rank as the times do."""
    return 12 * A.nnz + 4 * (A.nrows + 1) + 8 * A.ncols + 8 * A.nrows


def format_bytes(A, fmt):
    """The bytes a format must move by its own layout (padding excluded, x once),
    reported beside spmv_bytes: DIA stores no indices, 8 nnz + 8 ncols + 8 n;
    COO adds a row index per entry, 16 nnz + 8 ncols + 8 n; the other formats
    move what CSR moves."""
    if fmt.startswith("DIA"):
        return 8 * A.nnz + 8 * A.ncols + 8 * A.nrows
    if fmt.startswith("COO"):
        return 16 * A.nnz + 8 * A.ncols + 8 * A.nrows
    return spmv_bytes(A)


def cg_iteration_bytes(A, fmt=None):
    """Algorithmic bytes of one CG iteration: the SpMV plus 9 n-vector passes
    (read x, r, p, Ap and write x, r; read r, p and write p).  With ``fmt``, the
    SpMV counts the format's own bytes instead."""
    spmv = spmv_bytes(A) if fmt is None else format_bytes(A, fmt)
    return spmv + 9 * 8 * A.nrows


# DRAM traffic of the persistent CG kernel from one ncu capture (dram__bytes_read.sum
# + dram__bytes_write.sum over a launch that ran a known number of iterations:
# forced DIA, FP64, 3D Poisson 128^3, 429 iterations), per iteration.  Valid only
# for the kernel sources it was taken on: the bench reports null traffic once
# any of them changes (their SHA-256 differs).  The capture's summary is
# profiles/k_cg_persist_dia_poisson3d_128.md.
PERSIST_KERNEL_SOURCES = ("cg_persist.cu", "persist.cuh", "spmv_rows.cuh", "common.cuh")
PERSIST_TRAFFIC = {"format": "DIA", "n": 2097152,
                   "sha256": "b99f562a21c66ee044bae620a4b9c0ab79bf582404251e813823bf89545ca9b3",
                   "dram_bytes_per_iteration": 165605960.8}


def persist_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for name in PERSIST_KERNEL_SOURCES:
        h.update((ROOT / "paper_2411_10143_b300" / "csrc" / name).read_bytes())
    return h.hexdigest()


def persist_traffic(A, fmt, iters_per_launch):
    """DRAM bytes of one persistent launch from the recorded capture, or None."""
    t = PERSIST_TRAFFIC
    if (fmt != t["format"] or A.nrows != t["n"] or not t["sha256"]
            or persist_sources_sha256() != t["sha256"]):
        return None
    return t["dram_bytes_per_iteration"] * iters_per_launch


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ------------------------------------------------------------------ CPU oracle arms
REF_MAX_STEPS = 3  # full oracle solves the reference arm times (about 17 s each)


def host_cores():
    """Cores this process may run on (the host's nproc under its affinity mask)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_solve_ms(A, b, all_cores=False):
    """One full oracle CG solve of the benchmark system to 1e-10 from x0 = 0:
    (milliseconds, iterations, true relative residual, threads)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.cg_all_cores(A, b, tol=TOL) if all_cores else oracle.cg(A, b, tol=TOL)
    ms = (time.perf_counter() - t0) * 1e3
    return ms, r.iters, r.relres_true, (r.threads if all_cores else 1)


def run_reference(args, world, rank):
    """The CPU oracle as the reference arm: each timed step is one full
    single-threaded oracle CG solve of the benchmark system (no extrapolation).
    At most REF_MAX_STEPS steps are timed so that the arm ends within about a
    minute; the line's ``steps`` is the number actually run."""
    if rank != 0:
        return
    import oracle
    A, xs = workload()
    b = oracle.spmv(A, xs)
    for _ in range(args.warmup):  # warm the caches and the page tables: 5 iterations
        oracle.cg(A, b, tol=1e-300, maxit=5)
    steps = max(1, min(args.steps, REF_MAX_STEPS))
    t0 = time.perf_counter()
    runs = [oracle_solve_ms(A, b) for _ in range(steps)]
    region = time.perf_counter() - t0
    value = float(np.mean([r[0] for r in runs]))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ms",
        "n_gpus": args.gpus, "steps": steps, "steps_requested": args.steps,
        "warmup": args.warmup, "ms_per_step": region * 1e3 / steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(A),
        "cpu_baseline": {"value": value, "unit": "ms", "cores": 1, "kind": "oracle",
                         "host_cores": host_cores(),
                         "sample": f"{steps} full single-threaded oracle CG solves to "
                                   f"{TOL:g} ({runs[-1][1]} iterations, true relative "
                                   f"residual {runs[-1][2]:.2e}), no extrapolation"},
        "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_config(A):
    return {"workload": "CG, 3D 7-point Poisson 128^3 (n=2,097,152, nnz=14,581,760), FP64, "
                        "rel. residual 1e-10, asynchronous cascaded prediction on a side stream",
            "n": A.nrows, "nnz": A.nnz, "tol": TOL, "x0": "zeros", "rhs": "b = A x*, x* ~ U[-1,1]",
            "l2": "inputs larger than L2 (CSR 192 MB + 4 vectors of 16.8 MB vs 126 MB L2)"}


# ------------------------------------------------------------------ GPU arm
def run_ours(args, world, rank, local):
    import torch
    from paper_2411_10143_b300 import cascade as C
    from paper_2411_10143_b300 import models

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(local)
    torch.cuda.set_stream(stream)
    ctx = C.Context(local, main_stream=stream)
    loaded = models.load_default(ctx)
    ctx.warmup()  # every solve-path kernel launched once before any timing
    A, xs = workload()
    M = ctx.load(A)
    xs_d = torch.as_tensor(xs, device="cuda")
    b = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    M.spmv(xs_d, b)  # b = A x* by the library's default SpMV
    x = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
    opts = C.default_opts(tol=TOL, mode=C.MODE_ASYNC, profile=1, check_every=8)

    def step():
        M.reset()
        x.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = M.solve_cg(b, x, opts)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), info

    # the clock sampler runs from before the warm-up to the end of the timed
    # region, started early so that its own start-up is not timed
    with ClockSampler(local) as clk:
        clk.wait_first()
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        barrier(world)
        launches0 = ctx.launch_count()
        infos, tts = [], []
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        # an NVTX start/end range (it spans the side thread's launches too) marks
        # the timed steps, so a profiler's launch list can keep only their
        # kernels: ncu --nvtx --nvtx-include "timed steps"
        timed_range = torch.cuda.nvtx.range_start("timed steps")
        for _ in range(args.steps):
            ms, info = step()
            tts.append(ms)
            infos.append(info)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_end(timed_range)
        barrier(world)
        region = time.perf_counter() - t0
    gpu_launches = ctx.launch_count() - launches0
    value = max_over_ranks(float(np.mean(tts)), world, "cuda")
    region = max_over_ranks(region, world, "cuda")
    last = infos[-1]
    err = float(torch.linalg.norm(x - xs_d) / torch.linalg.norm(xs_d))

    # roofline of the dominant kernel, from CUDA events on the main stream inside
    # the timed solves: the persistent CG kernel running the predicted
    # configuration (its last launch in every solve), else the SpMV launches
    peak, peak_kind = measured_peaks()
    fmt = repr(last.final_cfg)
    t_last = sum(i.t_persist_last_ms for i in infos)
    it_last = sum(i.persist_last_iters for i in infos)
    n_spmv = sum(i.n_spmv for i in infos)
    t_spmv = sum(i.t_spmv_ms for i in infos)
    own = None
    if t_last > 0:
        kernel = f"k_cg_persist ({fmt}): one launch runs the CG iterations after the switch"
        per_launch = cg_iteration_bytes(A) * it_last / len(infos)
        launches = len(infos)
        avg_us = t_last / len(infos) * 1e3
        achieved = cg_iteration_bytes(A) * it_last / (t_last * 1e-3) / 1e9
        own = cg_iteration_bytes(A, fmt) * it_last / (t_last * 1e-3) / 1e9
        traffic = persist_traffic(A, fmt, it_last / len(infos))
    else:
        kernel = f"spmv ({fmt})"
        per_launch = spmv_bytes(A)
        launches = n_spmv
        avg_us = t_spmv / max(n_spmv, 1) * 1e3
        achieved = spmv_bytes(A) * n_spmv / (t_spmv * 1e-3) / 1e9 if t_spmv > 0 else None
        traffic = None
    extra = {}
    if rank == 0 and not args.no_compare:
        extra = comparisons(args, ctx, M, A, b, x, xs_d, stream, C)
    line = {
        "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": region * 1e3 / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(A),
        "roofline": {"bound": "hbm", "kernel": kernel,
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": traffic,
                     "peak_kind": peak_kind, "bytes_per_launch": per_launch,
                     "bytes": "12 nnz + 4 (n+1) + 16 n per SpMV (CSR matrix, x once, y once) "
                              "+ 9 x 8 n vector passes per CG iteration",
                     "launches": launches, "avg_launch_us": avg_us,
                     "achieved_own_format_bytes": own,
                     "frac_own_format_bytes": own / peak if own else None},
        "gpu_launches": int(gpu_launches),
        "clocks": clk.summary(),
        "solve": {"iters": last.iters, "final_cfg": repr(last.final_cfg),
                  "persist_iters": last.persist_iters, "t_persist_ms": last.t_persist_ms,
                  "switch_iter": list(last.switch_iter), "relres_true": last.relres_true,
                  "err_vs_xstar": err, "t_features_ms": last.t_features_ms,
                  "t_predict_ms": list(last.t_predict_ms), "t_convert_ms": last.t_convert_ms,
                  "models": loaded},
        "solves_per_s": world * args.steps / region,
    }
    line.update(extra)
    if "plain_csr_cg_ms" in line:
        line["speedup_vs_plain"] = line["plain_csr_cg_ms"] / value
        line["speedup_async_vs_sequential"] = line["sequential_ms"] / value
    if rank == 0:
        print(json.dumps(line), flush=True)


def comparisons(args, ctx, M, A, b, x, xs_d, stream, C):
    """Plain / sequential / FP32-IR variants, the end-to-end number, the CPU baseline."""
    import torch
    from paper_2411_10143_b300 import workloads as W

    def timed(opts, reps=2):
        out = []
        for _ in range(reps):
            M.reset()
            x.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = M.solve_cg(b, x, opts)
            e1.record(stream)
            e1.synchronize()
            out.append((e0.elapsed_time(e1), info))
        return float(np.mean([o[0] for o in out])), out[-1][1]

    plain_ms, plain = timed(C.default_opts(tol=TOL, mode=C.MODE_PLAIN))
    seq_ms, seq = timed(C.default_opts(tol=TOL, mode=C.MODE_SEQUENTIAL))
    ir_ms, ir = timed(C.default_opts(tol=TOL, mode=C.MODE_ASYNC, precision=C.PREC_FP32_IR,
                                     inner_tol=1e-5, ir_theta=IR_THETA))
    irf_ms, irf = timed(C.default_opts(tol=TOL, mode=C.MODE_ASYNC, precision=C.PREC_FP32_IR,
                                       inner_tol=1e-5, ir_theta=0.0))
    res = {
        "plain_csr_cg_ms": plain_ms, "plain_iters": plain.iters,
        "sequential_ms": seq_ms, "fp32_ir_async_ms": ir_ms,
        "fp32_ir": {"outer": ir.outer_iters, "inner": ir.iters, "relres_true": ir.relres_true,
                    "final_cfg": repr(ir.final_cfg), "inner_tol": 1e-5, "ir_theta": IR_THETA,
                    "every_inner_to_inner_tol": {"ms": irf_ms, "outer": irf.outer_iters,
                                                 "inner": irf.iters,
                                                 "relres_true": irf.relres_true}},
    }
    # end to end through host buffers: pinned CSR + b in, x out, per step
    rp = torch.as_tensor(A.rowptr).pin_memory()
    ci = torch.as_tensor(A.col).pin_memory()
    va = torch.as_tensor(A.val).pin_memory()
    bh = b.cpu().pin_memory()
    xh = torch.empty(A.nrows, dtype=torch.float64).pin_memory()
    opts = C.default_opts(tol=TOL, mode=C.MODE_ASYNC)
    e2e = []
    for k in range(5):  # one warm-up pass (first use of the load path), four timed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Mh = ctx.csr_load(A.nrows, A.ncols, rp.numpy(), ci.numpy(), va.numpy())
        bd = bh.to("cuda", non_blocking=True)
        xd = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
        Mh.solve_cg(bd, xd, opts)
        xh.copy_(xd, non_blocking=True)
        torch.cuda.synchronize()
        if k > 0:
            e2e.append((time.perf_counter() - t0) * 1e3)
        Mh.free()
    res["e2e"] = {"value": float(np.mean(e2e)), "unit": "ms",
                  "h2d_bytes_per_step": int(rp.numel() * 4 + ci.numel() * 4 + va.numel() * 8
                                            + bh.numel() * 8),
                  "d2h_bytes_per_step": int(xh.numel() * 8)}
    if not args.no_gmres:
        res["gmres"] = gmres_bench(ctx)
    if not args.no_sweep:
        res["spmv_sweep"] = spmv_sweep_bench(ctx, measured_peaks()[0], solves=True)
    if not args.no_gmres:
        # the random SPD power-law system of the asynchronous solves (n = 500k)
        res["spd_powerlaw_cg"] = variant_solves(ctx, W.spd_powerlaw(), W.RHS_SEED_BASE + 3, "cg")
        res["async_by_size"] = async_by_size(ctx)
    if args.serve_requests > 0:
        res["serve"] = serve_bench(ctx, args.serve_requests)
    if args.gpus == 1 and not args.no_cpu_baseline:
        # the oracle as it stands, one full solve, then its all-core build
        import oracle
        bn = b.cpu().numpy()
        ms1, it1, rel1, _ = oracle_solve_ms(A, bn)
        msn, itn, reln, thr = oracle_solve_ms(A, bn, all_cores=True)
        res["cpu_baseline"] = {
            "value": ms1, "unit": "ms", "cores": 1, "kind": "oracle", "host_cores": host_cores(),
            "sample": f"one full single-threaded oracle CG solve to {TOL:g} ({it1} iterations, "
                      f"true relative residual {rel1:.2e}), no extrapolation",
            "all_cores": {"value": msn, "unit": "ms", "threads": thr, "iters": itn,
                          "relres_true": reln,
                          "build": "the same oracle.c compiled with -fopenmp: row-parallel "
                                   "SpMV and CG vector loops, static-chunk reductions"}}
    return res


# ------------------------------------------------------------------ GMRES leg
GMRES_GRID = 96
GMRES_M = 30
# FP64 FMA lanes per second of the B300: 2 per SM per clock (148 SMs, 2,032 MHz)
FP64_DFMA_PEAK = 2 * 148 * 2.032e9


def gmres_dfma(n, nnz, iters, m):
    """Algorithmic FP64 FMAs of GMRES(m) with modified Gram-Schmidt over `iters`
    Arnoldi steps: step j of a cycle costs nnz (SpMV) + (j + 1) n dot products +
    (j + 1) n updates + n for the norm; a cycle of L steps adds L n for x += V y
    and nnz + n for the restart residual and its norm."""
    total, left = 0, iters
    while left > 0:
        L = min(m, left)
        total += L * nnz + n * (L * L + 2 * L) + L * n + nnz + n
        left -= L
    return total


def gmres_bench(ctx, reps=2):
    """GMRES(30) on convection-diffusion 96^3 (n = 884,736): the asynchronous
    cascade in FP64 and with FP32 inner solves, the one-launch-per-step CSR
    iteration, and the persistent kernel with DIA forced, whose FP64 FMA rate
    gives the roofline (the kernel is bound by the FP64 pipe)."""
    import torch
    from paper_2411_10143_b300 import cascade as C
    from paper_2411_10143_b300 import workloads as W

    A = W.convdiff3d(GMRES_GRID)
    M = ctx.load(A)
    xs = torch.as_tensor(W.vector(A.ncols, 2004), device="cuda")
    b = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    M.spmv(xs, b)
    x = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")

    def timed(opts, force=None, reset=True):
        ts, info = [], None
        for _ in range(reps):
            if reset:
                M.reset()
            x.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            info = M.solve_gmres(b, x, opts, force=force)
            e1.record(ctx.stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.mean(ts)), info

    base = dict(tol=TOL, restart=GMRES_M)
    # the metric's denominator: plain FP64 GMRES on the default CSR-scalar
    # kernel, on the library's default iteration path (the persistent kernel)
    plain_ms, pl = timed(C.default_opts(mode=C.MODE_PLAIN, **base))
    async_ms, a = timed(C.default_opts(mode=C.MODE_ASYNC, **base))
    ir_ms, ir = timed(C.default_opts(mode=C.MODE_ASYNC, precision=C.PREC_FP32_IR,
                                     inner_tol=1e-5, ir_theta=IR_THETA, **base))
    irf_ms, irf = timed(C.default_opts(mode=C.MODE_ASYNC, precision=C.PREC_FP32_IR,
                                       inner_tol=1e-5, ir_theta=0.0, **base))
    step_ms, st = timed(C.default_opts(mode=C.MODE_PLAIN, iteration_kernel=1, **base))
    dia = C.config("DIA")
    M.convert(dia)
    dia_ms, d = timed(C.default_opts(mode=C.MODE_PLAIN, **base), force=dia, reset=False)
    flops = gmres_dfma(A.nrows, A.nnz, d.persist_iters, GMRES_M)
    rate = flops / (d.t_persist_ms * 1e-3)
    peak = ctx.fp64_fma_rate()
    return {
        "workload": f"GMRES({GMRES_M}), convection-diffusion {GMRES_GRID}^3 (n={A.nrows:,}, "
                    f"nnz={A.nnz:,}), FP64, rel. residual {TOL:g}, b = A x*, x0 = 0",
        "plain_csr_gmres_ms": plain_ms, "plain_iters": pl.iters,
        "plain_relres_true": pl.relres_true,
        "async_ms": async_ms, "iters": a.iters, "final_cfg": repr(a.final_cfg),
        "relres_true": a.relres_true, "persist_iters": a.persist_iters,
        "fp32_ir_async_ms": ir_ms, "fp32_ir": {"outer": ir.outer_iters, "inner": ir.iters,
                                               "relres_true": ir.relres_true,
                                               "inner_tol": 1e-5, "ir_theta": IR_THETA,
                                               "every_inner_to_inner_tol": {
                                                   "ms": irf_ms, "outer": irf.outer_iters,
                                                   "inner": irf.iters,
                                                   "relres_true": irf.relres_true}},
        "csr_scalar_one_launch_per_step_ms": step_ms, "one_launch_per_step_launches":
            st.n_launches,
        "persistent_dia_ms": dia_ms,
        "speedup_vs_plain": {"async": plain_ms / async_ms, "fp32_ir_async": plain_ms / ir_ms,
                             "dia_forced": plain_ms / dia_ms},
        "roofline": {"kernel": "k_gm_persist (DIA, FP64, modified Gram-Schmidt)", "bound": "alu",
                     "achieved": rate / 1e9, "peak": peak / 1e9,
                     "unit": "G FP64 FMA/s", "frac": rate / peak,
                     "fma_per_solve": flops, "peak_kind": "measured",
                     "peak_note": "cp_fp64_fma_rate: independent FMA chains on every SM, best "
                                  "of five launches; nominal 2 per SM per clock x 148 SMs x "
                                  f"2,032 MHz = {FP64_DFMA_PEAK / 1e9:.1f}"},
    }


# ------------------------------------------------------------------ serving leg
def sweep_configs(C):
    """Every SpMV configuration of the format space (Sec. III-B-2, Table III)."""
    cfgs = [C.config("CSR", algo=C.ALGO_SCALAR)]
    cfgs += [C.config("CSR", algo=C.ALGO_VECTOR, tpv=t) for t in (2, 4, 8, 16, 32)]
    cfgs += [C.config("CSR", algo=C.ALGO_MERGE), C.config("COO"), C.config("ELL")]
    cfgs += [C.config("SELL", sigma=s) for s in (1, 32, 1024, 8192)]
    cfgs += [C.config("HYB"), C.config("DIA")]
    return cfgs


def time_spmv(ctx, M, cfg, x, y, reps, warm):
    """Median and mean of reps back-to-back launches (CUDA events around each,
    on the library's stream), after warm launches.  The matrices are larger
    than L2, so every launch streams them from HBM."""
    import torch
    for _ in range(warm):
        M.spmv(x, y, cfg)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    torch.cuda.synchronize()
    for e0, e1 in ev:
        e0.record(ctx.stream)
        M.spmv(x, y, cfg)
        e1.record(ctx.stream)
    torch.cuda.synchronize()
    t = np.array([e0.elapsed_time(e1) for e0, e1 in ev])
    return float(np.median(t)), float(np.mean(t))


def timed_solve(ctx, M, b, xstar, kind, opts, force=None, reps=2):
    """Mean time (CUDA events on the library's stream) of `reps` solves from x0 = 0,
    every one from the freshly loaded CSR (converted formats and features dropped),
    with the last solve's info and its error against x*."""
    import torch
    ts, info, x = [], None, None
    for _ in range(reps):
        M.reset()
        x = torch.zeros(M.nrows, dtype=torch.float64, device="cuda")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        info = (M.solve_cg if kind == "cg" else M.solve_gmres)(b, x, opts, force=force)
        e1.record(ctx.stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    err = float(torch.linalg.norm(x - xstar) / torch.linalg.norm(xstar))
    return float(np.mean(ts)), info, err


def variant_solves(ctx, A, seed, kind, restart=30):
    """A solve on a matrix: plain FP64 with the default CSR-scalar kernel against
    the asynchronous cascade with FP32 inner solves in FP64 refinement (and in
    FP64 for CG), to relative residual 1e-10; b = A x*."""
    import torch
    from paper_2411_10143_b300 import cascade as C
    from paper_2411_10143_b300 import workloads as W
    M = ctx.load(A)
    xs = torch.as_tensor(W.vector(A.ncols, seed), device="cuda")
    b = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    M.spmv(xs, b)
    base = dict(tol=TOL, restart=restart)
    out = {"n": A.nrows, "nnz": A.nnz}
    legs = [("plain_fp64", C.default_opts(mode=C.MODE_PLAIN, **base))]
    if kind == "cg":
        legs.append(("async_fp64", C.default_opts(mode=C.MODE_ASYNC, **base)))
    legs.append(("async_fp32_ir", C.default_opts(mode=C.MODE_ASYNC, precision=C.PREC_FP32_IR,
                                                 inner_tol=1e-5, **base)))
    for name, opts in legs:
        # the plain leg once: on the power-law variant CSR-scalar takes tens of seconds
        ms, info, err = timed_solve(ctx, M, b, xs, kind, opts, reps=1 if name == "plain_fp64" else 2)
        out[name] = {"ms": ms, "iters": info.iters, "outer": info.outer_iters,
                     "final_cfg": repr(info.final_cfg), "relres_true": info.relres_true,
                     "err_vs_xstar": err, "switch_iter": list(info.switch_iter),
                     "persist_iters": info.persist_iters,
                     "t_persist_ms": round(float(info.t_persist_ms), 3),
                     "t_features_ms": round(float(info.t_features_ms), 3),
                     "t_predict_ms": round(float(sum(info.t_predict_ms)), 3),
                     "t_convert_ms": round(float(info.t_convert_ms), 3)}
    out["speedup_vs_plain"] = out["plain_fp64"]["ms"] / out["async_fp32_ir"]["ms"]
    M.free()
    return out


def async_by_size(ctx, grids=(24, 32, 48, 64, 96, 128), reps=5, log_fn=log):
    """Where asynchrony pays (Sec. III-C-2, Table VII): FP64 CG to 1e-10 on 3D
    Poisson systems of several sizes, plain (CSR-scalar throughout), sequential
    (prediction and conversion first, then the predicted kernel) and
    asynchronous (the solve starts at once on CSR-scalar and switches when the
    prediction lands); medians of ``reps`` solves each, every one from the
    freshly loaded CSR.  The cascade's side work costs about the same at every
    size, so its share, and what overlapping it saves, grows as the solve
    shortens."""
    import torch
    from paper_2411_10143_b300 import cascade as C
    from paper_2411_10143_b300 import workloads as W
    out = {}
    for N in grids:
        A = W.poisson3d(N)
        M = ctx.load(A)
        xs = torch.as_tensor(W.vector(A.ncols, XSTAR_SEED), device="cuda")
        b = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
        M.spmv(xs, b)
        row = {"n": A.nrows}
        for name, mode in (("plain", C.MODE_PLAIN), ("sequential", C.MODE_SEQUENTIAL),
                           ("async", C.MODE_ASYNC)):
            ts, info = [], None
            for _ in range(reps):
                ms, info, _ = timed_solve(ctx, M, b, xs, "cg", C.default_opts(tol=TOL, mode=mode),
                                          reps=1)
                ts.append(ms)
            row[f"{name}_ms"] = float(np.median(ts))
            if name == "async":
                row["async_switch_iter"] = list(info.switch_iter)
                row["iters"] = info.iters
                row["final_cfg"] = repr(info.final_cfg)
                row["gate_declined"] = info.gate_declined
        row["async_vs_sequential"] = row["sequential_ms"] / row["async_ms"]
        row["async_vs_plain"] = row["plain_ms"] / row["async_ms"]
        out[f"poisson3d_{N}"] = row
        log_fn(f"async by size: 3D Poisson {N}^3 plain {row['plain_ms']:.2f} ms, sequential "
               f"{row['sequential_ms']:.2f} ms, async {row['async_ms']:.2f} ms")
        M.free()
    return out


def spmv_sweep_bench(ctx, peak, reps=200, warm=10, only_predicted=False, log_fn=log,
                     solves=False, matrices=None, config=None):
    """SpMV format/kernel sweep with cascaded prediction on the four sweep
    matrices (3D Poisson 128^3, power law, uniform, banded; FP64 values
    U[-1,1]): per matrix the predicted configuration's GB/s and fraction of the
    measured HBM peak, the best and the CSR-scalar configuration beside it, and
    the cost of the prediction (features + three stages) and of the conversion.
    GB/s counts algorithmic bytes (padding excluded, x once).  ``matrices``
    (names) and ``config`` (a configuration name such as "ELL" or "CSR-merge",
    with only_predicted) narrow it for profiling."""
    import torch
    from paper_2411_10143_b300 import cascade as C
    from paper_2411_10143_b300 import workloads as W
    out = {}
    for k, (name, gen) in enumerate(W.spmv_sweep().items()):
        if matrices and name not in matrices:
            continue
        A = gen()
        M = ctx.load(A)
        x = torch.as_tensor(W.vector(A.ncols, W.RHS_SEED_BASE + 1), device="cuda")
        y = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cfg_p, stage_ms = M.predict()
        t_pred = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        M.convert(cfg_p)
        torch.cuda.synchronize()
        t_conv = (time.perf_counter() - t0) * 1e3
        if config:
            cfg_p = next(c for c in sweep_configs(C) if repr(c) == config)
        cfgs = [cfg_p] if only_predicted else sweep_configs(C)
        if repr(cfg_p) not in [repr(c) for c in cfgs]:
            cfgs.append(cfg_p)
        rows = {}
        for cfg in cfgs:
            try:
                M.convert(cfg)
            except C.CascadeError as e:  # padded format over its memory budget, DIA > 1024 offsets
                rows[repr(cfg)] = {"skipped": str(e)[:80]}
                continue
            med, mean = time_spmv(ctx, M, cfg, x, y, reps, warm)
            gbs = spmv_bytes(A) / (med * 1e-3) / 1e9
            own = format_bytes(A, repr(cfg)) / (med * 1e-3) / 1e9
            rows[repr(cfg)] = {"median_us": med * 1e3, "mean_us": mean * 1e3, "gbs": gbs,
                               "frac": gbs / peak, "gbs_own_format_bytes": own,
                               "frac_own_format_bytes": own / peak}
        timed = {c: r for c, r in rows.items() if "median_us" in r}
        best = min(timed, key=lambda c: timed[c]["median_us"])
        pr = rows[repr(cfg_p)]
        res = {"n": A.nrows, "nnz": A.nnz, "predicted": repr(cfg_p), "predicted_gbs": pr["gbs"],
               "predicted_frac": pr["frac"], "predict_ms": t_pred, "predict_stage_ms":
               [float(v) for v in stage_ms], "convert_ms": t_conv}
        if not only_predicted:
            base = rows["CSR-scalar"]
            res.update({"best": best, "best_gbs": timed[best]["gbs"], "best_frac": timed[best]["frac"],
                        "csr_scalar_gbs": base["gbs"],
                        "speedup_vs_csr_scalar": base["median_us"] / pr["median_us"],
                        "regret": pr["median_us"] / timed[best]["median_us"], "configs": rows})
        if solves and name != "poisson3d":
            # the mixed-precision solve on this matrix's nonsymmetric solve variant
            # (the same pattern, diagonally dominant), GMRES(30)
            res["gmres_variant"] = variant_solves(ctx, W.diagonally_dominant(A),
                                                  W.RHS_SEED_BASE + 4, "gmres")
        out[name] = res
        log_fn(f"spmv sweep {name}: predicted {res['predicted']} {pr['gbs']:.0f} GB/s "
               f"({pr['frac']:.2f} of peak)" + ("" if only_predicted else
               f", best {best} {timed[best]['gbs']:.0f} GB/s"))
        M.free()
        del x, y
    return out


def serve_bench(ctx, count, seed=3000, lanes=4, log_fn=log):
    """Continuous-batching server under Poisson arrivals: n log-uniform in
    [1e3, 1e6], 40 % 2D/3D Poisson (CG), 30 % SPD power law (CG), 30 %
    convection-diffusion (GMRES(30)), FP32 inner solves in FP64 refinement to
    1e-10.  The stream is replayed at 0.5, 0.8, 1.0, 1.2 and 2.0 x the sequential
    (one-lane) service rate measured on a sample of the same requests (0.8 x gives the
    headline p50 / p99), once with every request submitted at once (the
    saturation throughput), and once served one request at a time by plain FP64
    CSR-scalar solves at 0.8 x (the baseline).  Matrices are generated once per
    size bucket (6 per decade and kind) and stay resident; every request has its
    own right-hand side."""
    import torch
    from paper_2411_10143_b300 import cascade as C
    from paper_2411_10143_b300 import workloads as W
    reqs = W.request_stream(count=count, rate_per_s=1.0, seed=seed)
    buckets = {}

    def bucket(r):
        kb = (r.kind, int(round(np.log10(r.n) * 6)))
        if kb not in buckets:
            n = int(round(10 ** (kb[1] / 6)))
            A = W.request_matrix(W.Request(0, 0.0, r.kind, n, seed + kb[1]))
            buckets[kb] = (A, ctx.load(A))
        return buckets[kb]

    t0 = time.time()
    items = []
    for r in reqs:
        A, M = bucket(r)
        xs = torch.as_tensor(W.vector(A.nrows, r.seed % 100000), device="cuda")
        b = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
        M.spmv(xs, b)
        items.append((r, A, M, 1 if r.kind == "convdiff" else 0, b))
    torch.cuda.synchronize()
    log_fn(f"serve: {len(buckets)} resident matrices built in {time.time() - t0:.0f}s")
    # the batching autotuner on three random groups of small requests (the
    # classes the server's batches fall in); cp_batch_solve then uses its picks
    rng = np.random.default_rng(seed + 1)
    small = [it for it in items if it[1].nrows <= 32768]
    tuned = []
    for _ in range(3 if len(small) >= 32 else 0):
        grp = [small[i] for i in rng.choice(len(small), 32, replace=False)]
        bopts = C.default_opts(tol=TOL, inner_tol=1e-5, restart=30, precision=C.PREC_FP32_IR)
        best, ms, (order, ms_order) = ctx.batch_tune([g[2] for g in grp], [g[3] for g in grp],
                                                     [g[4] for g in grp], bopts, with_order=True)
        # the same batch at the tuned block size with every system's threads per
        # row from the BATCH_TPR classifier (the server's default), launch time
        # as the tuner measures it (median of three after one warm-up)
        per = []
        for _ in range(4):
            xs = [torch.zeros(g[1].nrows, dtype=torch.float64, device="cuda") for g in grp]
            infos = ctx.batch_solve([g[2] for g in grp], [g[3] for g in grp],
                                    [g[4] for g in grp], xs, bopts, best[0], 0)
            per.append(infos[0].t_total_ms)
        picks = [ctx.batch_tpr(g[2]) for g in grp]
        tuned.append({"mean_rows": int(np.mean([g[1].nrows for g in grp])),
                      "gmres": any(g[3] for g in grp), "threads": best[0],
                      "threads_per_row": best[1],
                      "ms": {f"{t}x{r}": round(v, 3) for (t, r), v in ms.items()},
                      "packing_order": "caller's order" if order else "largest first",
                      "caller_order_ms": round(ms_order, 3),
                      "per_system_classifier_ms": round(float(np.median(per[1:])), 3),
                      "per_system_threads_per_row": {str(r): picks.count(r) for r in (1, 4, 16)}})
    log_fn(f"serve: batch autotuner picks {[(t['threads'], t['threads_per_row']) for t in tuned]}, "
           f"tuned {[round(min(t['ms'].values()), 2) for t in tuned]} ms, per-system classifier "
           f"{[t['per_system_classifier_ms'] for t in tuned]} ms")
    # sequential service rate on a sample
    srv = C.Server(ctx, lanes=1)
    sample = items[: min(24, len(items))]
    t1 = time.perf_counter()
    for k, (r, A, M, s, b) in enumerate(sample):
        x = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
        srv.submit(k, M, s, b, x)
        srv.drain(600)
    seq = (time.perf_counter() - t1) / len(sample)
    srv.poll()
    srv.close()
    out = {"requests": len(items), "sequential_service_ms": seq * 1e3, "lanes": lanes,
           "resident_matrices": len(buckets), "batch_tuning": tuned, "loads": {}}
    for load in SERVE_LOADS:
        res = serve_replay(ctx, items, load / seq, lanes, C)
        res["load"] = load
        out["loads"][f"{load:g}"] = res
        log_fn(f"serve at {load:g}x: p50 {res['p50_ms']:.1f} ms, p99 {res['p99_ms']:.1f} ms, "
               f"{res['solves_per_s']:.1f} solves/s (offered {res['arrival_rate_per_s']:.1f})")
    sat = serve_replay(ctx, items, None, lanes, C)
    out["saturation"] = sat
    log_fn(f"serve, every request at once: {sat['solves_per_s']:.1f} solves/s")
    plain = serve_plain(ctx, items, 0.8 / seq, C)
    out["plain_one_at_a_time"] = plain
    log_fn(f"serve, plain FP64 CSR-scalar one at a time at 0.8x: p50 {plain['p50_ms']:.1f} ms, "
           f"p99 {plain['p99_ms']:.1f} ms")
    # the headline figures: the 0.8x load
    main = out["loads"]["0.8"]
    for k in ("p50_ms", "p99_ms", "solves_per_s", "arrival_rate_per_s", "completed_ok",
              "batched", "max_relres_true", "failures"):
        out[k] = main[k]
    out["saturation_solves_per_s"] = sat["solves_per_s"]
    return out


SERVE_LOADS = (0.5, 0.8, 1.0, 1.2, 2.0)  # arrival rate / sequential service rate


def serve_replay(ctx, items, rate, lanes, C):
    """Replay the requests' arrivals at ``rate`` per second (None: all at once)
    into a server with ``lanes`` lanes; latency is arrival to completion."""
    import torch
    srv = C.Server(ctx, lanes=lanes)
    xs_keep = []
    start = time.perf_counter()
    for k, (r, A, M, s, b) in enumerate(items):
        if rate is not None:
            due = start + r.arrival_s / rate
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                time.sleep(min(due - now, 0.002))
        x = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
        xs_keep.append(x)
        srv.submit(k, M, s, b, x)
    srv.drain(1800)
    wall = time.perf_counter() - start
    res = srv.poll(capacity=len(items) + 8)
    srv.close()
    lat = np.array([q.t_done_ms - q.t_submit_ms for q in res])
    fails = [{"id": int(q.id), "kind": items[q.id][0].kind, "n": int(items[q.id][1].nrows),
              "status": int(q.status), "relres": q.relres_true, "batched": int(q.batched)}
             for q in res if q.status != 0][:10]
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "solves_per_s": len(res) / wall,
            "arrival_rate_per_s": rate if rate is not None else None,
            "completed_ok": sum(1 for q in res if q.status == 0),
            "batched": int(sum(q.batched for q in res)),
            "max_relres_true": max(q.relres_true for q in res) if res else None,
            "failures": fails}


def serve_plain(ctx, items, rate, C):
    """The same arrivals served one request at a time by plain FP64 solves on
    the default CSR-scalar kernel (the library's default iteration path, no
    prediction, no batching): the baseline the served solve is compared with.
    Latency is arrival to completion; a request waits while the one before it
    runs."""
    import torch
    opts = C.default_opts(tol=TOL, mode=C.MODE_PLAIN, restart=30)
    lat, worst, ok = [], 0.0, 0
    start = time.perf_counter()
    for r, A, M, s, b in items:
        due = start + r.arrival_s / rate
        while True:
            now = time.perf_counter()
            if now >= due:
                break
            time.sleep(min(due - now, 0.002))
        x = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
        info = (M.solve_gmres if s else M.solve_cg)(b, x, opts, raise_on_error=False)
        torch.cuda.current_stream().synchronize()
        lat.append((time.perf_counter() - due) * 1e3)
        ok += info.status == 0
        worst = max(worst, info.relres_true)
    wall = time.perf_counter() - start
    lat = np.array(lat)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "solves_per_s": len(items) / wall, "arrival_rate_per_s": rate, "completed_ok": ok,
            "max_relres_true": worst}


def run_profile_cg(args):
    """One configuration, no prediction: plain-mode CG on the bench workload with
    the SpMV configuration forced, so the persistent kernel runs every iteration
    in one launch (the case the profiles under profiles/ capture).  Prints one
    JSON line per solve; not a bench line."""
    import torch
    from paper_2411_10143_b300 import cascade as C

    ctx = C.Context(0)
    if args.profile_matrix == "spd_powerlaw":
        from paper_2411_10143_b300 import workloads as W
        A = W.spd_powerlaw()
        xs = W.vector(A.ncols, W.RHS_SEED_BASE + 3)
    else:
        A, xs = workload()
    M = ctx.load(A)
    xs_d = torch.as_tensor(xs, device="cuda")
    b = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    M.spmv(xs_d, b)
    cfg = C.config(args.profile_cg)
    M.convert(cfg)
    opts = C.default_opts(tol=TOL, mode=C.MODE_PLAIN, precision=args.profile_precision, profile=1)
    for k in range(args.steps):
        x = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        info = M.solve_cg(b, x, opts, force=cfg)
        e1.record(ctx.stream)
        e1.synchronize()
        print(json.dumps({"solve": k, "config": repr(cfg), "precision": args.profile_precision,
                          "ms": e0.elapsed_time(e1), "iters": info.iters,
                          "persist_iters": info.persist_iters, "t_persist_ms": info.t_persist_ms,
                          "us_per_iteration": info.t_persist_ms * 1e3 / max(info.persist_iters, 1),
                          "relres_true": info.relres_true}), flush=True)


def run_profile_gmres(args):
    """Forced-configuration GMRES(30) solves on the GMRES leg's workload
    (convection-diffusion 96^3), plain mode, so one persistent launch runs the
    whole solve (the case the GMRES profile under profiles/ captures).  Prints
    one JSON line per solve; not a bench line."""
    import torch
    from paper_2411_10143_b300 import cascade as C
    from paper_2411_10143_b300 import workloads as W

    ctx = C.Context(0)
    A = W.convdiff3d(GMRES_GRID)
    M = ctx.load(A)
    xs = torch.as_tensor(W.vector(A.ncols, 2004), device="cuda")
    b = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    M.spmv(xs, b)
    cfg = C.config(args.profile_gmres)
    M.convert(cfg)
    opts = C.default_opts(tol=TOL, mode=C.MODE_PLAIN, restart=GMRES_M,
                          precision=args.profile_precision, inner_tol=1e-5)
    for k in range(args.steps):
        x = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        info = M.solve_gmres(b, x, opts, force=cfg)
        e1.record(ctx.stream)
        e1.synchronize()
        print(json.dumps({"solve": k, "config": repr(cfg), "precision": args.profile_precision,
                          "ms": e0.elapsed_time(e1), "iters": info.iters,
                          "persist_iters": info.persist_iters, "t_persist_ms": info.t_persist_ms,
                          "us_per_step": info.t_persist_ms * 1e3 / max(info.persist_iters, 1),
                          "relres_true": info.relres_true}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving leg (0 skips it)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the plain / sequential / FP32-IR / end-to-end / CPU legs")
    ap.add_argument("--no-sweep", action="store_true", help="skip the SpMV sweep leg")
    ap.add_argument("--no-gmres", action="store_true", help="skip the GMRES leg")
    ap.add_argument("--profile-spmv", action="store_true",
                    help="profiling aid: the predicted SpMV of each sweep matrix, 3 launches")
    ap.add_argument("--spmv-matrix", default=None,
                    help="with --profile-spmv: sweep matrices to run (comma-separated names)")
    ap.add_argument("--spmv-config", default=None,
                    help="with --profile-spmv: run this configuration (e.g. ELL, CSR-merge) "
                         "instead of the predicted one")
    ap.add_argument("--profile-cg", default=None, metavar="FMT",
                    help="profiling aid: forced-configuration CG solves (e.g. DIA), no bench line")
    ap.add_argument("--profile-matrix", default="poisson3d", choices=["poisson3d", "spd_powerlaw"],
                    help="--profile-cg's system: the bench's 3D Poisson, or the SPD power law "
                         "(n 500k) of the spd_powerlaw_cg leg")
    ap.add_argument("--profile-precision", type=int, default=0,
                    help="with --profile-cg: 0 FP64, 1 FP32 inner solves in FP64 refinement")
    ap.add_argument("--profile-gmres", default=None, metavar="FMT",
                    help="profiling aid: forced-configuration GMRES(30) solves on "
                         "convection-diffusion 96^3, no bench line")
    args = ap.parse_args()
    if args.profile_cg:
        run_profile_cg(args)
        return
    if args.profile_gmres:
        run_profile_gmres(args)
        return
    if args.profile_spmv:
        from paper_2411_10143_b300 import cascade as C
        from paper_2411_10143_b300 import models
        ctx = C.Context(0)
        models.load_default(ctx)
        print(json.dumps(spmv_sweep_bench(
            ctx, measured_peaks()[0], reps=3, warm=1, only_predicted=True,
            matrices=args.spmv_matrix.split(",") if args.spmv_matrix else None,
            config=args.spmv_config)), flush=True)
        return
    if args.impl == "reference":
        world, rank, _ = dist_init("gloo")
        run_reference(args, world, rank)
        return
    world, rank, local = dist_init("nccl")
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
