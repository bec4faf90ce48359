"""Benchmark: block PLHR seconds to k interior pairs at relative residual 1e-8.

Workload: 3D 7-point Dirichlet Laplacian on a 128^3 grid (n = 2,097,152,
h = 1/129), sigma midway between the eigenvalues 1064.022 and 1073.120
(index ~471), k = 10 wanted pairs (k' = 11 columns, real arithmetic),
preconditioner = 4-level AV-MG V-cycle with 2 pre/post smoothing steps.
A step is one complete solve from the seeded starting block to
convergence (all k relative residuals <= 1e-8 after the final Rayleigh-Ritz).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision f64]

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
# the traffic grows in proportion to n m (profiles/k_gram_lap3d_64cube.md).
GRAM_DRAM_BYTES_PER_ROW_COL = 446.1e6 / (262144 * 64)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
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
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _vcycle_bytes(n, ncols, levels):
    """Algorithmic HBM bytes of one V-cycle on ncols FP64 columns: the finest
    level reads r and writes w once per smoothing step (2 nu sweeps) plus the
    residual/restriction pass, i.e. about 6 column passes, and every coarser
    level adds 1/8 of that."""
    per_level = 6 * n * ncols * 8
    return per_level * sum(0.125 ** l for l in range(levels))


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1408_0042_gb300 as plhr
    import workloads as wl

    torch.cuda.set_device(local)
    w = wl.config2()
    profile_case = args.profile_grid > 0
    if profile_case:
        # reduced grid with the same structure, a fixed number of iterations:
        # the case the ncu captures run on
        N = args.profile_grid
        w = dataclasses.replace(w, name="lap3d_%dcube_k10_%dit" % (N, args.profile_iters), dims=(N, N, N),
                                h=1.0 / (N + 1), maxit=args.profile_iters,
                                mg_levels=max(1, int(round(math.log2(N / 16)))) + 1)
    n, k, kp = w.n, w.k, w.kprime
    t_setup = time.perf_counter()
    A = plhr.Operator.laplacian(w.dims, w.h)
    T = plhr.AVMG(A, w.sigma, levels=w.mg_levels, nu=w.mg_nu, transfer=MG_TRANSFER, coarse=MG_COARSE)
    v0_host = torch.from_numpy(w.v0()).pin_memory()
    v0 = v0_host.cuda()
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream()

    def one(vinit):
        return plhr.solve(A, w.sigma, k, T=T, tol=w.tol, maxit=w.maxit, v_init=vinit,
                          raise_on_notconv=not profile_case, guard=w.guard)

    for _ in range(args.warmup):
        lam, V, info = one(v0)
    torch.cuda.synchronize()
    iters = info["iterations"]

    # ---------------------------------------------------------------- timed region
    plhr.profile_read(reset=True)
    plhr.profile_enable(True)
    launches0 = plhr.kernel_launches()
    times = []
    with ClockSampler(local) as clk:
        _barrier(world)
        torch.cuda.synchronize()
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
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
    clocks = clk.summary()
    step_s = _max_over_ranks(statistics.mean(times), world)
    iters = info["iterations"]

    if profile_case:
        if rank == 0:
            print(json.dumps({"profile_case": w.name, "seconds": step_s, "iterations": iters,
                              "gpu_launches": launches,
                              "phases_ms": {p: prof[p]["ms"] / max(1, args.steps) for p in prof}}), flush=True)
        return
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
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vdev = v0_host.to("cuda", non_blocking=True)
        lam2, V2, _ = one(vdev)
        vecs_host.copy_(V2, non_blocking=True)
        vals_host.copy_(torch.from_numpy(lam2))
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1) / 1e3)
    e2e_s = _max_over_ranks(statistics.mean(e2e_times), world)

    # ---------------------------------------------------------------- roofline of the dominant phase
    peaks = _peaks()
    dom = max(("preconditioner", "gram", "update", "stencil"), key=lambda p: prof[p]["ms"])
    m_avg = kp + 2 * kp + kp   # trial basis size of a full iteration
    if dom == "gram":
        flops = 2.0 * n * (m_avg * (m_avg + 1) / 2 + 2 * m_avg * m_avg)
        per = prof["gram"]["ms"] / max(1, prof["gram"]["calls"]) / 1e3
        achieved = flops / per / 1e12
        roof = {"kernel": "k_gram (FP64 multi-Gram Z^T Z, U^T Q, Q^T Z)", "bound": "alu",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": GRAM_DRAM_BYTES_PER_ROW_COL * n * m_avg,
                "traffic_note": "ncu dram bytes of k_gram on the 64^3 case scaled by n m",
                "peak_src": "nominal FP64 rate of the profiling recipe"}
    elif dom == "update":
        flops = 3 * 2.0 * n * (m_avg * kp + kp * kp)
        per = prof["update"]["ms"] / max(1, prof["update"]["calls"]) / 1e3
        achieved = flops / per / 1e12
        roof = {"kernel": "k_update x3 (FP64 coefficient update)", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_src": "nominal FP64 rate of the profiling recipe"}
    else:
        calls = max(1, prof[dom]["calls"])
        cols = (kp + 2 * kp + kp) / 3.0
        byt = _vcycle_bytes(n, cols, w.mg_levels) if dom == "preconditioner" else 3 * n * kp * 8
        per = prof[dom]["ms"] / calls / 1e3
        achieved = byt / per / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_src": peaks["src"]}

    out = {
        "metric": METRIC, "value": step_s, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded start block)",
        "config": {"workload": w.name, "operator": "7-point Dirichlet Laplacian 128^3, h = 1/129",
                   "n": n, "k": k, "k_prime": kp, "sigma": w.sigma, "tol": w.tol,
                   "preconditioner": {"kind": "AV-MG", "levels": w.mg_levels, "nu": w.mg_nu,
                                      "transfer": "trilinear", "coarse": "fine-spectrum"},
                   "l2": "inputs larger than L2 (one 128^3 x 11 FP64 block = 185 MB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "iterations": iters, "setup_s": setup_s, "max_rel_residual": info["max_rel_residual"],
        "max_rel_eig_err_vs_closed_form": eig_err,
        "fp64_seconds": step_s, "mixed_seconds": None,
        "phases_ms_per_step": {p: prof[p]["ms"] / max(1, args.steps) for p in prof},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": n * kp * 8,
                "d2h_bytes_per_step": n * k * 8 + k * 8},
        "gpu_launches": launches, "roofline": roof, "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(iters)
    if rank == 0:
        print(json.dumps(out), flush=True)


def _oracle_iteration_seconds(samples=1):
    """Time the FP64 oracle on the 128^3 workload: setup, then `samples`
    iterations (the per-iteration work is the same at every iteration)."""
    import numpy as np

    import workloads as wl
    from oracle import avmg, operators, plhr

    w = wl.config2()
    A, _ = operators.model_operator(w)
    T = avmg.AVMG(w.dims, w.h, w.sigma, w.mg_levels, w.mg_nu, transfer="linear", coarse="fine_spectrum")
    marks = []
    t0 = time.perf_counter()
    plhr.bplhr(A, None, T, w.sigma, w.k, w.v0(), tol=w.tol, maxit=samples,
               callback=lambda rec: marks.append(time.perf_counter()))
    # marks[0]: after the start block and iteration-0 residual; marks[i]: after iteration i
    per = (marks[-1] - marks[0]) / max(1, len(marks) - 1)
    return per, time.perf_counter() - t0


def cpu_baseline(gpu_iterations):
    per, total = _oracle_iteration_seconds(samples=1)
    cores = os.cpu_count()
    return {"value": per * gpu_iterations, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": "1 oracle iteration of the 128^3 workload (%.1f s/iteration, %.1f s with setup), "
                      "scaled by the GPU iteration count %d" % (per, total, gpu_iterations)}


def run_reference(args, world, rank, local):
    if rank != 0:
        return
    import workloads as wl
    w = wl.config2()
    iters = w.extra.get("iterations_to_tol", 305)
    for _ in range(args.warmup):
        _oracle_iteration_seconds(samples=1)
    vals = []
    for _ in range(args.steps):
        per, _ = _oracle_iteration_seconds(samples=1)
        vals.append(per * iters)
    v = statistics.mean(vals)
    out = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded start block)", "impl": "reference",
           "config": {"workload": w.name, "n": w.n, "k": w.k, "tol": w.tol},
           "cpu_baseline": {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": "per step: 1 oracle iteration of the 128^3 workload, scaled by %d "
                                      "iterations to tolerance" % iters},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["f64"], default="f64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-grid", type=int, default=0,
                    help="profiling case: N^3 grid of the same problem, fixed iteration count")
    ap.add_argument("--profile-iters", type=int, default=3)
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
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1 and args.impl == "ours":
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
