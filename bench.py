"""Benchmark: block PLHR seconds to k interior pairs at relative residual 1e-8.

Workload: 3D 7-point Dirichlet Laplacian on a 128^3 grid (n = 2,097,152,
h = 1/129), sigma midway between the eigenvalues 1064.022 and 1073.120
(index ~471), k = 10 wanted pairs (k' = 16 block columns: 6 guard columns so
that the 1073.12 sextet and the 1080.75 sextet behind it fit the block, real
arithmetic), preconditioner = 4-level AV-MG V-cycle with 2 pre/post smoothing
steps.  A step is one complete solve from the seeded starting block to
convergence (all k relative residuals <= 1e-8 after the final Rayleigh-Ritz),
by default in the mixed-precision form (FP32 blocks and V-cycles until the k
residuals reach 1e-6, then FP64); one all-FP64 solve is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision mixed|f64] [--no-f64-compare]

One JSON line is printed by rank 0.  Under torchrun (N > 1) every rank solves
its own replica (the problem does not shard on one-GPU machines: replicas only)
and the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PLHR seconds to k interior pairs at rel. residual 1e-8, mixed vs FP64; HBM GB/s"

# Transfer and coarsest-operator reading of the AV-MG used for this workload
# (trilinear cell-centred transfers, coarsest operator with the fine-grid
# spectrum); the piecewise-constant / rediscretised reading does not converge
# on this grid.
MG_TRANSFER = 1
MG_COARSE = 1


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": p.get("hbm_gbs", 6800.0), "bf16_tflops": p.get("bf16_tflops", 1900.0),
                "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}


# FP64 rate of GB300 from the profiling recipe's nominal table (1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 1.25

# ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_gram launch on the
# 64^3 case (n = 262,144, m = 64): 446.1 MB, i.e. bytes per (row x trial column);
# the traffic grows in proportion to n m.
GRAM_DRAM_BYTES_PER_ROW_COL = 446.1e6 / (262144 * 64)
# the same for the double-word Gram k_gram_dw (m = 64 launch on the 64^3
# case: 402.8 MB read + 3.8 MB written)
GRAM_DW_DRAM_BYTES_PER_ROW_COL = 406.60e6 / (262144 * 64)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        # a GPU UUID ("GPU-...") names the device this process uses even when
        # CUDA_VISIBLE_DEVICES renumbers the devices; a plain index is the
        # fallback
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm), "gpu": str(self.index)}


def _gpu_id(local):
    """nvidia-smi's name of this process's GPU: its UUID ("GPU-..."), which
    stays right when CUDA_VISIBLE_DEVICES renumbers the devices; the local
    index if the UUID cannot be read."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(local)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(x, world):
    """Maximum of x over the ranks (NCCL between GPUs; a gloo group reduces
    on the host)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _vcycle_bytes_per_element(levels, elem_bytes):
    """Algorithmic HBM bytes of the V-cycle schedule per finest-level element
    (grid point x column): on each smoothing level the fused first two sweeps
    (read r, write w: 2 passes), the residual (3), the restriction (1 + 1/8),
    the prolongation with correction (2 + 1/8) and two post-sweeps (6), i.e.
    14.25 passes, each coarser level 1/8 of the one above (the coarsest solve
    is a few KB per column)."""
    return 14.25 * elem_bytes * sum(0.125 ** l for l in range(max(1, levels - 1)))


def _fp32_simt_peak_tflops(sm_mhz):
    """FP32 CUDA-core peak: 152 SMs x 128 FMA lanes x 2 flops x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


PHASE_KERNELS = {
    "stencil": "k_lap_axpby / k_lap_shifts (FP64) and k_lap32 (FP32) stencil products",
    "preconditioner": "AV-MG V-cycle kernels (FP64 form; double-word in the mixed form's FP64 phase)",
    "gram": "k_gram (FP64 multi-Gram; k_gram_dw double-word in the mixed form's FP64 phase)",
    "update": "k_update (FP64; k_update_dw double-word in the mixed form's FP64 phase)",
    "residual": "k_residual (residual block and column norms)",
    "preconditioner_f32": "FP32 AV-MG V-cycle kernels",
    "gram_f32": "k_gram_tc (tcgen05 multi-Gram, split-BF16 slices)",
    "update_f32": "k_update_mx (FP32 with double-word V part)",
}


def _rooflines(prof, peaks, sm_max_mhz, mixed, tensor_cores=True):
    """Achieved HBM bandwidth of every profiled phase: the library's
    algorithmic bytes (every operand block read once, every result written
    once per call) over its CUDA-event time, against the measured copy
    bandwidth.  Phases whose arithmetic also bounds them carry the ALU or
    tensor rate as a second figure: the double-word multiply-add costs 13
    FP32 instructions for 2 FP64-equivalent flops (roof = FP32 lane rate / 13),
    the FP64 kernels run at the FP64 rate of the profiling recipe, and the
    tensor-core Gram executes six BF16 slice products per useful product."""
    out = []
    fp32_peak = _fp32_simt_peak_tflops(sm_max_mhz or 2070.0)
    dw_peak = fp32_peak / 13.0
    alu = {
        "gram": ("double-word FP32-pipe roof" if mixed else "FP64 rate", dw_peak if mixed else FP64_PEAK_TFLOPS, 1.0),
        "update": ("double-word FP32-pipe roof" if mixed else "FP64 rate", dw_peak if mixed else FP64_PEAK_TFLOPS,
                   1.0),
        "gram_f32": (("BF16 tensor rate (6 slice products per product)", peaks["bf16_tflops"], 6.0) if tensor_cores
                     else ("FP32 lanes x clock", fp32_peak, 1.0)),
        "update_f32": ("FP32 lanes x clock", fp32_peak, 1.0),
    }
    kernels = dict(PHASE_KERNELS)
    if not tensor_cores:
        kernels["gram_f32"] = "k_gram_mx (FP32 products on the FP32 pipes, compensated sums)"
    for ph, d in prof.items():
        if ph == "dense" or not d or d["ms"] <= 0 or d.get("bytes", 0) <= 0:
            continue
        gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
        e = {"phase": ph, "kernel": kernels.get(ph, ph), "bound": "hbm", "achieved": gbs,
             "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
             "total_ms": d["ms"], "calls": d["calls"], "bytes_per_call": d["bytes"] / max(1, d["calls"]),
             "peak_src": "%s (MEASURED_PEAKS.json hbm_gbs)" % peaks["src"]}
        if ph in alu and d["work"] > 0:
            name, peak, mult = alu[ph]
            a = d["work"] * mult * 1e-12 / (d["ms"] / 1e3)
            e["alu"] = {"achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak, "roof": name}
        out.append(e)
    return sorted(out, key=lambda r: -r["total_ms"])


def lap3d_config(w, precision, switch_tol, parallelism):
    """The JSON config of the 128^3 Laplacian workload (both arms)."""
    return {"workload": w.name, "operator": "7-point Dirichlet Laplacian 128^3, h = 1/129",
            "n": w.n, "k": w.k, "k_prime": w.kprime, "sigma": w.sigma, "tol": w.tol, "precision": precision,
            "switch_tol": switch_tol if precision == "mixed" else None,
            "preconditioner": {"kind": "AV-MG", "levels": w.mg_levels, "nu": w.mg_nu,
                               "transfer": "trilinear", "coarse": "fine-spectrum"},
            "l2": "inputs larger than L2 (one 128^3 x 16 FP64 block = 268 MB)",
            "parallelism": parallelism}


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1408_0042_gb300 as plhr
    import workloads as wl

    torch.cuda.set_device(local)
    w = wl.lap3d_128cube_k10()
    profile_case = args.profile_grid > 0
    if profile_case:
        # reduced grid with the same structure, a fixed number of iterations:
        # the case the ncu captures run on
        N = args.profile_grid
        w = dataclasses.replace(w, name="lap3d_%dcube_k10_%dit" % (N, args.profile_iters), dims=(N, N, N),
                                h=1.0 / (N + 1), maxit=args.profile_iters,
                                mg_levels=max(1, int(round(math.log2(N / 16)))) + 1)
    n, k, kp = w.n, w.k, w.kprime
    prec = {"mixed": plhr.PRECISION_MIXED, "f64": plhr.PRECISION_F64}[args.precision]
    t_setup = time.perf_counter()
    A = plhr.Operator.laplacian(w.dims, w.h)
    T = plhr.AVMG(A, w.sigma, levels=w.mg_levels, nu=w.mg_nu, transfer=MG_TRANSFER, coarse=MG_COARSE)
    v0_host = torch.from_numpy(w.v0()).pin_memory()
    v0 = v0_host.cuda()
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream()

    def one(vinit, p=prec):
        return plhr.solve(A, w.sigma, k, T=T, tol=w.tol, maxit=w.maxit, v_init=vinit,
                          raise_on_notconv=not profile_case, guard=w.guard, precision=p,
                          switch_tol=args.switch_tol, tensor_cores=args.tensor_cores)

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    for _ in range(args.warmup):
        lam, V, info = one(v0)
    torch.cuda.synchronize()

    # ---------------------------------------------------------------- timed region
    plhr.profile_read(reset=True)
    plhr.profile_enable(True)
    launches0 = plhr.kernel_launches()
    times = []
    with ClockSampler(_gpu_id(local)) as clk:
        _barrier(world)
        torch.cuda.synchronize()
        for _ in range(args.steps):
            (lam, V, info), dt = timed(lambda: one(v0))
            times.append(dt)
        torch.cuda.synchronize()
        _barrier(world)
    launches = plhr.kernel_launches() - launches0
    plhr.profile_enable(False)
    prof = plhr.profile_read(reset=True)
    clocks = clk.summary()
    step_s = _max_over_ranks(statistics.mean(times), world)
    iters = info["iterations"]

    if profile_case:
        if rank == 0:
            print(json.dumps({"profile_case": w.name, "precision": args.precision, "seconds": step_s,
                              "iterations": iters, "gpu_launches": launches,
                              "phases_ms": {p: prof[p]["ms"] / max(1, args.steps) for p in prof}}), flush=True)
        return

    # the all-FP64 form on the same input, for the mixed-vs-FP64 comparison
    fp64_s, fp64_iters = None, None
    if args.precision == "mixed" and not args.no_f64_compare:
        (_, _, info64), fp64_s = timed(lambda: one(v0, plhr.PRECISION_F64))
        fp64_s = _max_over_ranks(fp64_s, world)
        fp64_iters = info64["iterations"]

    # closed-form check of the returned eigenvalues
    cf = wl.lap_closed_form(w.dims, w.h)
    want = np.sort(cf[np.lexsort((cf, np.abs(cf - w.sigma)))][:k])
    eig_err = float(np.abs(np.sort(lam) - want).max() / np.abs(want).max())

    # ---------------------------------------------------------------- end to end (host buffers)
    e2e_times = []
    vals_host = torch.empty(k, dtype=torch.float64).pin_memory()
    vecs_host = torch.empty((n, k), dtype=torch.float64).pin_memory()
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()

        def e2e_step():
            vdev = v0_host.to("cuda", non_blocking=True)
            lam2, V2, _ = one(vdev)
            vecs_host.copy_(V2, non_blocking=True)
            vals_host.copy_(torch.from_numpy(lam2))
        _, dt = timed(e2e_step)
        e2e_times.append(dt)
    e2e_s = _max_over_ranks(statistics.mean(e2e_times), world)

    # ---------------------------------------------------------------- rooflines
    peaks = _peaks()
    roofs = _rooflines(prof, peaks, clocks.get("sm_max_mhz"), args.precision == "mixed", args.tensor_cores)
    dom = dict(roofs[0]) if roofs else None
    if dom is not None:
        dom["traffic"] = None
        if dom["phase"] == "gram":
            # ncu DRAM bytes per (row x trial column) of the kernel, scaled to the
            # average launch of this run (the algorithmic bytes are 3 n m x 8)
            per = GRAM_DRAM_BYTES_PER_ROW_COL if args.precision == "f64" else GRAM_DW_DRAM_BYTES_PER_ROW_COL
            m_avg = dom["bytes_per_call"] / (24.0 * n)
            dom["traffic"] = per * n * m_avg
            dom["traffic_note"] = ("ncu dram__bytes_read + write of one %s launch with m = 64 on the 64^3 case, "
                                   "scaled by n m to this run's average launch (n = %d, m = %.1f)" % (
                                       "k_gram" if args.precision == "f64" else "k_gram_dw", n, m_avg))
    dense = prof.get("dense", {})
    dense_stage = {"ms_per_iteration": dense["ms"] / dense["calls"] if dense.get("calls") else None,
                   "ms_per_step": dense.get("ms", 0.0) / max(1, args.steps),
                   "bound": "latency (m <= 64 projected problem on the device, no HBM traffic)"}

    out = {
        "metric": METRIC, "value": step_s, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic (seeded start block)",
        "config": lap3d_config(w, args.precision, args.switch_tol,
                               "replicas" if world > 1 else "single GPU"),
        "iterations": iters, "mixed_iterations": info.get("mixed_iterations", 0), "setup_s": setup_s,
        "max_rel_residual": info["max_rel_residual"], "max_rel_eig_err_vs_closed_form": eig_err,
        "mixed_seconds": step_s if args.precision == "mixed" else None,
        "fp64_seconds": step_s if args.precision == "f64" else fp64_s, "fp64_iterations": fp64_iters,
        "phases_ms_per_step": {p: prof[p]["ms"] / max(1, args.steps) for p in prof},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": n * kp * 8,
                "d2h_bytes_per_step": n * k * 8 + k * 8},
        "gpu_launches": launches, "roofline": dom, "rooflines": roofs[1:], "dense_stage": dense_stage,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(fp64_iters or iters, "FP64" if fp64_iters else args.precision)
    if rank == 0:
        print(json.dumps(out), flush=True)


class _OracleCase:
    """The FP64 oracle's operator and AV-MG for the 128^3 workload (built once)."""

    def __init__(self):
        import workloads as wl
        from oracle import avmg, operators
        t0 = time.perf_counter()
        self.w = wl.lap3d_128cube_k10()
        self.A, _ = operators.model_operator(self.w)
        self.T = avmg.AVMG(self.w.dims, self.w.h, self.w.sigma, self.w.mg_levels, self.w.mg_nu,
                           transfer="linear", coarse="fine_spectrum")
        self.v0 = self.w.v0()
        self.setup_s = time.perf_counter() - t0

    def steady_iteration(self):
        """Time one steady-state oracle iteration: the second one, the first
        whose trial basis holds P (m = 4 k'); the first (m = 3 k') runs
        untimed.  Returns (seconds, host cores busy on average = process CPU
        time / wall time of the timed iteration)."""
        from oracle import plhr
        marks = []

        def cb(rec):
            marks.append((time.perf_counter(), time.process_time()))
        w = self.w
        plhr.bplhr(self.A, None, self.T, w.sigma, w.k, self.v0, tol=w.tol, maxit=2, callback=cb)
        # marks[i]: start of iteration i (after its residual); iteration 1 = marks[1] -> marks[2]
        (w1, c1), (w2, c2) = marks[1], marks[2]
        return w2 - w1, (c2 - c1) / max(w2 - w1, 1e-9)


def cpu_baseline(iterations, which):
    case = _OracleCase()
    per, cores = case.steady_iteration()
    return {"value": per * iterations, "unit": "s", "cores": round(cores, 1), "kind": "oracle",
            "sample": "1 steady-state oracle iteration of the 128^3 workload (the second, m = 4k' = 64: %.1f s; "
                      "setup %.1f s), scaled by the GPU's %s iteration count %d; cores = CPU time / wall time "
                      "of that iteration (%d host cores present)" % (per, case.setup_s, which, iterations,
                                                                    os.cpu_count())}


LAP2D_METRIC = "PLHR seconds to k interior pairs at rel. residual 1e-8 (FP64)"


def run_lap2d(args, world, rank, local):
    """The small 2D workload: 5-point Dirichlet Laplacian on 32 x 32 interior
    points (n = 1024, h = 1/33), the 4 pairs nearest sigma = 1297.84 (the
    midpoint of lambda_100 and lambda_101, closed form), T = I, FP64, tol 1e-8,
    guard 2 (the double eigenvalue outside the wanted set).  A step is one
    solve from the seeded start block.  Latency-bound at this size: every
    iteration is a few dozen small launches and one host synchronisation."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1408_0042_gb300 as plhr
    import workloads as wl

    torch.cuda.set_device(local)
    w = wl.lap2d_32x32_k4()
    A = plhr.Operator.laplacian(w.dims, w.h)
    v0_host = torch.from_numpy(w.v0()).pin_memory()
    v0 = v0_host.cuda()
    stream = torch.cuda.current_stream()

    def one(vinit):
        return plhr.solve(A, w.sigma, w.k, tol=w.tol, maxit=w.maxit, v_init=vinit, guard=w.guard,
                          raise_on_notconv=True)

    for _ in range(args.warmup):
        one(v0)
    torch.cuda.synchronize()
    plhr.profile_read(reset=True)
    plhr.profile_enable(True)
    launches0 = plhr.kernel_launches()
    times = []
    with ClockSampler(_gpu_id(local)) as clk:
        _barrier(world)
        torch.cuda.synchronize()
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lam, V, info = one(v0)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        _barrier(world)
    launches = plhr.kernel_launches() - launches0
    plhr.profile_enable(False)
    prof = plhr.profile_read(reset=True)
    step_s = _max_over_ranks(statistics.mean(times), world)
    cf = wl.lap_closed_form(w.dims, w.h)
    want = np.sort(cf[np.lexsort((cf, np.abs(cf - w.sigma)))][: w.k])
    eig_err = float(np.abs(np.sort(lam) - want).max() / np.abs(want).max())
    e2e = []
    vecs_host = torch.empty((w.n, w.k), dtype=torch.float64).pin_memory()
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lam2, V2, _ = one(v0_host.to("cuda", non_blocking=True))
        vecs_host.copy_(V2, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e.append(e0.elapsed_time(e1) / 1e3)
    e2e_s = _max_over_ranks(statistics.mean(e2e), world)
    roofs = _rooflines(prof, _peaks(), clk.summary().get("sm_max_mhz"), False)
    out = {
        "metric": LAP2D_METRIC, "value": step_s, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded start block)",
        "config": {"workload": w.name, "operator": "5-point Dirichlet Laplacian 32 x 32, h = 1/33", "n": w.n,
                   "k": w.k, "k_prime": w.kprime, "sigma": w.sigma, "tol": w.tol, "preconditioner": "none (T = I)",
                   "l2": "the whole problem fits in L2 (latency-bound)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "iterations": info["iterations"], "max_rel_residual": info["max_rel_residual"],
        "max_rel_eig_err_vs_closed_form": eig_err, "us_per_iteration": step_s / max(1, info["iterations"]) * 1e6,
        "phases_ms_per_step": {p: prof[p]["ms"] / max(1, args.steps) for p in prof},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": w.n * w.kprime * 8,
                "d2h_bytes_per_step": w.n * w.k * 8},
        "gpu_launches": launches, "roofline": roofs[0] if roofs else None, "rooflines": roofs[1:],
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import operators, plhr as oplhr
        Ao, _ = operators.model_operator(w)
        t0, c0 = time.perf_counter(), time.process_time()
        r = oplhr.bplhr(Ao, None, None, w.sigma, w.k, w.v0(), tol=w.tol, maxit=w.maxit)
        t1, c1 = time.perf_counter(), time.process_time()
        out["cpu_baseline"] = {"value": t1 - t0, "unit": "s", "cores": round((c1 - c0) / max(t1 - t0, 1e-9), 1),
                               "kind": "oracle",
                               "sample": "the full oracle solve of the same workload (%d iterations); cores = CPU "
                                         "time / wall time (%d host cores present)" % (r.iterations, os.cpu_count())}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_gram_case(args, world, rank, local):
    """The projected-Gram pass on its own (rows A6 of the hot path): every
    arithmetic form of plhr_gram on seeded random families shaped like one
    m = 64 launch of the mixed form (Z, AZ, Q as four blocks of 16 columns; Q
    a positive row scaling of U = AZ - sigma Z, so that U^T Q is symmetric as
    in the solver), n = --gram-case rows; CUDA events around each call (which
    also allocates its partial-sum buffer on the stream and reads back one
    status word).  Reports ms per call and the algorithmic bytes 3 n m x
    element size over that time."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1408_0042_gb300 as plhr

    torch.cuda.set_device(local)
    n, ncols, sigma = args.gram_case, [16, 16, 16, 16], 1068.5711114200
    m = sum(ncols)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(20140801)
    res = {}
    peaks = _peaks()
    for form in [int(f) for f in args.gram_forms.split(",")]:
        dt = torch.float64 if form in (plhr.GRAM_F64, plhr.GRAM_DW) else torch.float32
        Z = [torch.randn(n, c, dtype=dt, device="cuda", generator=gen) for c in ncols]
        A = [sigma * torch.randn(n, c, dtype=dt, device="cuda", generator=gen) for c in ncols]
        wts = 1e-3 * (0.5 + torch.rand(n, 1, dtype=dt, device="cuda", generator=gen))
        Q = [(wts * (a - sigma * z)).contiguous() for z, a in zip(Z, A)]
        cs = torch.ones(m, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            plhr.gram(form, Z, A, Q, sigma, cs)
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plhr.gram(form, Z, A, Q, sigma, cs)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        gbs = 3.0 * n * m * (8 if dt == torch.float64 else 4) / (ms / 1e3) / 1e9
        res[{0: "f64", 1: "f32_pipes", 2: "double_word", 3: "f32_tensor_cores"}[form]] = {
            "ms_per_call": ms, "GB_per_s": gbs, "frac_of_hbm": gbs / peaks["hbm_gbs"]}
        del Z, A, Q
        torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps({"gram_case": {"n": n, "m": m, "steps": args.steps, "warmup": args.warmup,
                                        "peak_hbm_gbs": peaks["hbm_gbs"], "forms": res}}), flush=True)


GRAD_METRIC = ("seconds per forward + backward: k = 8 eigenpairs nearest sigma and dL/dV of "
               "sum_k w_k lambda_k + sum_k |m (.) v_k|^2, 64^3 Hamiltonian")


def run_grad(args, world, rank, local):
    """The differentiation workload: a step is the forward solve (TPA-
    preconditioned block PLHR, FP64, tol 1e-10) plus the backward pass
    (eigenvalue gradient and the eigenvector adjoint) for one potential."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1408_0042_gb300 as plhr
    import workloads as wl

    torch.cuda.set_device(local)
    c = wl.ham64_k8_grad()
    dims, sigma, k = c["dims"], c["sigma"], c["k"]
    n = int(np.prod(dims))
    guard, tol, adj_tol = 2, 1e-10, 1e-10
    kp = k + guard
    V_host = torch.from_numpy(c["V"]).pin_memory()
    Vd = V_host.cuda()
    v0 = torch.from_numpy(wl.start_block(n, kp, c["seed"])).cuda()
    wt = torch.from_numpy(c["w"]).cuda()
    mt = torch.from_numpy(c["mask"]).cuda()
    adj_prec = args.adjoint_prec

    def step(Vdev):
        op = plhr.Operator.hamiltonian(dims, 1.0, Vdev)
        T = plhr.TPA(op, sigma)
        lam, vecs, info = plhr.solve(op, sigma, k, T=T, tol=tol, maxit=2000, guard=guard, v_init=v0,
                                     raise_on_notconv=True)
        order = np.argsort(lam)                      # w attaches to the eigenvalues in ascending order
        wk = np.empty(k)
        wk[order] = c["w"]
        g = plhr.eigval_grad(vecs, wk)
        G = (2.0 * mt[:, None] * vecs).contiguous()  # dL/dv_k of the density term
        ga, its = plhr.eigvec_adjoint(op, lam, vecs, G, tol=adj_tol, T=T if adj_prec == "tpa" else None,
                                      return_iterations=True)
        g += ga
        loss = float(np.dot(wk, lam)) + float((mt[:, None] * vecs * vecs).sum())
        return g, lam, info, its, loss

    def timed_parts(Vdev):
        # forward and backward times of one step (CUDA events on the stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        op = plhr.Operator.hamiltonian(dims, 1.0, Vdev)
        T = plhr.TPA(op, sigma)
        lam, vecs, info = plhr.solve(op, sigma, k, T=T, tol=tol, maxit=2000, guard=guard, v_init=v0)
        ev[1].record(stream)
        G = (2.0 * mt[:, None] * vecs).contiguous()
        plhr.eigval_grad(vecs, np.ones(k))
        plhr.eigvec_adjoint(op, lam, vecs, G, tol=adj_tol, T=T if adj_prec == "tpa" else None)
        ev[2].record(stream)
        ev[2].synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3

    for _ in range(args.warmup):
        step(Vd)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    plhr.profile_read(reset=True)
    plhr.profile_enable(True)
    launches0 = plhr.kernel_launches()
    times = []
    with ClockSampler(_gpu_id(local)) as clk:
        _barrier(world)
        torch.cuda.synchronize()
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g, lam, info, its, loss = step(Vd)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        _barrier(world)
    launches = plhr.kernel_launches() - launches0
    plhr.profile_enable(False)
    prof = plhr.profile_read(reset=True)
    clocks = clk.summary()
    step_s = _max_over_ranks(statistics.mean(times), world)

    fwd_s, bwd_s = timed_parts(Vd)
    # check of the answer: the 8 nearest eigenvalues from a Lanczos solve of
    # the oracle's operator (workloads/select_shift_ham64.py)
    lam_ref = np.array(wl.HAM64_LAMBDA_REF)
    eig_err = float(np.abs(np.sort(lam) - lam_ref).max())

    # end to end: V from pinned host memory, the gradient back to the host
    g_host = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Vdev = V_host.to("cuda", non_blocking=True)
        g2, _, _, _, _ = step(Vdev)
        g_host.copy_(g2, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    e2e_s = _max_over_ranks(statistics.mean(e2e), world)

    # rooflines of the phases the library times; the TPA application is dense
    # per-axis transforms in double-word arithmetic: 2 (forward, inverse) x 2
    # flops x (nx + ny + nz) per element (grid point x column)
    fp64 = FP64_PEAK_TFLOPS
    dw_peak = _fp32_simt_peak_tflops(clocks.get("sm_max_mhz") or 2070.0) / 13.0
    per_elem = 4.0 * sum(dims)
    roofs = []
    for ph, kernel, per, peak, src in (
            ("preconditioner", "k_axis (TPA transforms, double-word)", per_elem * 1e-12, dw_peak,
             "FP32 lanes x clock / 13 x 2 flops (double-word multiply-add = 13 FP32 instructions)"),
            ("gram", "k_gram (FP64 multi-Gram)", 1e-12, fp64, "nominal FP64 rate of the profiling recipe"),
            ("update", "k_update (FP64)", 1e-12, fp64, "nominal FP64 rate of the profiling recipe")):
        d = prof.get(ph)
        if not d or d["ms"] <= 0 or d["work"] <= 0:
            continue
        a = d["work"] * per / (d["ms"] / 1e3)
        roofs.append({"phase": ph, "kernel": kernel, "bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s",
                      "frac": a / peak, "total_ms": d["ms"], "calls": d["calls"], "traffic": None,
                      "peak_src": src})
    roofs.sort(key=lambda r: -r["total_ms"])
    out = {
        "metric": GRAD_METRIC, "value": step_s, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded potential and start block)",
        "config": {"workload": "ham64_k8_grad", "operator": "-1/2 Lap + V, 64^3 periodic, h = 1, 32 Gaussian wells",
                   "n": n, "k": k, "k_prime": kp, "sigma": sigma, "tol": tol, "adjoint_tol": adj_tol,
                   "preconditioner": "TPA (forward)" + (", TPA (adjoint)" if adj_prec == "tpa" else ""),
                   "l2": "inputs larger than L2 (the 9 n x k adjoint blocks and the 64 n x k' trial blocks)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "iterations": info["iterations"], "adjoint_iterations": its, "max_rel_residual": info["max_rel_residual"],
        "max_abs_eig_err_vs_lanczos": eig_err, "forward_s": fwd_s, "backward_s": bwd_s, "loss": loss,
        "phases_ms_per_step": {p: prof[p]["ms"] / max(1, args.steps) for p in prof},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
        "gpu_launches": launches, "roofline": roofs[0] if roofs else None, "rooflines": roofs[1:],
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = grad_cpu_baseline(info["iterations"])
    if rank == 0:
        print(json.dumps(out), flush=True)


def grad_cpu_baseline(gpu_iterations):
    """The oracle's forward solve of the 64^3 workload (TPA by FFT), one
    iteration timed and scaled by the GPU iteration count.  The oracle's
    adjoint is the full-spectrum formula (a dense eigendecomposition of the
    262,144 x 262,144 operator), so the backward pass has no CPU baseline."""
    import numpy as np

    import workloads as wl
    from oracle import operators, plhr, spectral

    c = wl.ham64_k8_grad()
    H = operators.hamiltonian(c["dims"], 1.0, c["V"])
    T = spectral.TPA(c["dims"], 1.0, spectral.default_energy(c["sigma"], c["V"], c["dims"], 1.0))
    n = H.shape[0]
    marks = []
    t0 = time.perf_counter()
    plhr.bplhr(H, None, T, c["sigma"], c["k"], wl.start_block(n, c["k"] + 2, c["seed"]), tol=1e-10, maxit=1,
               callback=lambda rec: marks.append(time.perf_counter()))
    per = (marks[-1] - marks[0]) / max(1, len(marks) - 1)
    return {"value": per * gpu_iterations, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "1 oracle iteration of the forward solve (%.1f s/iteration, %.1f s with setup), scaled by "
                      "the GPU iteration count %d; forward only" % (per, time.perf_counter() - t0, gpu_iterations)}


# Iterations of the all-FP64 GPU form to relative residual 1e-8 on the 128^3
# workload (293, measured on GB300 by this bench's fp64 leg); the oracle runs
# the same FP64 iteration, and its own count would take over an hour of host
# time to measure, so the reference arm scales its per-iteration time by the
# GPU's count.
GPU_F64_ITERATIONS_TO_TOL = 293


def run_reference(args, world, rank, local):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.
    Each timed step runs the oracle's first two iterations of the 128^3
    workload and times the second (steady state, m = 4k'), scaled by the GPU
    FP64 iteration count to tolerance; a warm-up step runs the start block
    and first residual only.  Under torchrun only rank 0 runs and prints; the
    other ranks return at once."""
    if rank != 0:
        return
    from oracle import plhr as oplhr
    case = _OracleCase()
    w = case.w
    iters = GPU_F64_ITERATIONS_TO_TOL
    for _ in range(args.warmup):
        oplhr.bplhr(case.A, None, case.T, w.sigma, w.k, case.v0, tol=w.tol, maxit=0)
    vals, cores = [], []
    for _ in range(args.steps):
        per, c = case.steady_iteration()
        vals.append(per * iters)
        cores.append(c)
    v = statistics.mean(vals)
    out = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded start block)", "impl": "reference",
           "config": lap3d_config(w, "f64", None, "host cores (FP64 oracle)"),
           "cpu_baseline": {"value": v, "unit": "s", "cores": round(statistics.mean(cores), 1), "kind": "oracle",
                            "sample": "per step: the oracle's second (steady-state, m = 4k') iteration of the "
                                      "128^3 workload, scaled by the GPU FP64 iteration count %d; cores = CPU "
                                      "time / wall time (%d host cores present)" % (iters, os.cpu_count())},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "f64"], default="mixed")
    ap.add_argument("--switch-tol", type=float, default=1e-6,
                    help="mixed form: residual level where the FP32 phase hands over to the double-word phase")
    ap.add_argument("--no-f64-compare", action="store_true",
                    help="skip the all-FP64 solve timed beside the mixed-precision steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tensor-cores", dest="tensor_cores", action="store_false",
                    help="mixed form: FP32-phase Grams on the FP32 pipes instead of the tensor cores")
    ap.add_argument("--profile-grid", type=int, default=0,
                    help="profiling case: N^3 grid of the same problem, fixed iteration count")
    ap.add_argument("--profile-iters", type=int, default=3)
    ap.add_argument("--workload", choices=["lap3d_128cube_k10", "ham64_k8_grad", "lap2d_32x32_k4"],
                    default="lap3d_128cube_k10",
                    help="ham64_k8_grad: forward + backward of the 64^3 differentiation workload; "
                         "lap2d_32x32_k4: the 32 x 32 Laplacian, T = I, FP64")
    ap.add_argument("--gram-case", type=int, default=0,
                    help="time plhr_gram alone on random families of n = GRAM_CASE rows, m = 64")
    ap.add_argument("--gram-forms", default="0,1,2,3",
                    help="with --gram-case: forms to time (0 FP64, 1 FP32 pipes, 2 double-word, 3 tensor cores)")
    ap.add_argument("--adjoint-prec", choices=["none", "tpa"], default="none",
                    help="preconditioner of the adjoint MINRES in the ham64_k8_grad workload")
    args = ap.parse_args()
    world, rank, local = _dist()
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        if args.impl == "reference":
            run_reference(args, world, rank, local)
        elif args.gram_case > 0:
            run_gram_case(args, world, rank, local)
        elif args.workload == "ham64_k8_grad":
            run_grad(args, world, rank, local)
        elif args.workload == "lap2d_32x32_k4":
            run_lap2d(args, world, rank, local)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1 and args.impl == "ours":
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
