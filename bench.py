"""Benchmark: block PLHR seconds to k interior pairs at relative residual 1e-8.

Workload: 3D 7-point Dirichlet Laplacian on a 128^3 grid (n = 2,097,152,
h = 1/129), sigma midway between the eigenvalues 1064.022 and 1073.120
(index ~471), k = 10 wanted pairs (k' = 16 block columns: 6 guard columns so
that the 1073.12 sextet and the 1080.75 sextet behind it fit the block, real
arithmetic), preconditioner = 4-level AV-MG V-cycle with 2 pre/post smoothing
steps.  A step is one complete solve from the seeded starting block to
convergence (all k relative residuals <= 1e-8 after the final Rayleigh-Ritz),
by default in the mixed-precision form (FP32 blocks and V-cycles until the k
residuals reach 1e-5, then FP64); one all-FP64 solve is timed beside it.

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
# the traffic grows in proportion to n m (profiles/k_gram_lap3d_64cube.md).
GRAM_DRAM_BYTES_PER_ROW_COL = 446.1e6 / (262144 * 64)
# the same for the double-word Gram k_gram_dw (m = 64 launch on the 64^3
# case: 402.8 MB read + 3.8 MB written; profiles/mixed_form_kernels_lap3d_64cube.md)
GRAM_DW_DRAM_BYTES_PER_ROW_COL = 406.60e6 / (262144 * 64)


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


def _rooflines(prof, w, peaks, sm_max_mhz, mixed):
    """Achieved rate of every profiled phase from its algorithmic work and its
    CUDA-event time; returns the entries sorted by total time.  In the mixed
    form the FP64 phase runs the Gram, the update and the V-cycle in
    double-word arithmetic on FP32 pipes: a double-word multiply-add costs 13
    FP32 instructions (lane operations) for 2 FP64-equivalent flops, so its
    compute roof is (FP32 lane operations per second) x 2 / 13 = the FP32
    flop rate / 13."""
    out = []
    fp32_peak = _fp32_simt_peak_tflops(sm_max_mhz or 2070.0)
    dw_peak = fp32_peak / 13.0
    if mixed:
        f64_rows = [("gram", "k_gram_dw (double-word multi-Gram)", "alu", dw_peak, "TFLOP/s", 1e-12),
                    ("update", "k_update_dw (double-word update)", "alu", dw_peak, "TFLOP/s", 1e-12),
                    ("preconditioner", "double-word AV-MG V-cycle kernels", "hbm", peaks["hbm_gbs"], "GB/s",
                     _vcycle_bytes_per_element(w.mg_levels, 8) * 1e-9)]
    else:
        f64_rows = [("gram", "k_gram (FP64 multi-Gram)", "alu", FP64_PEAK_TFLOPS, "TFLOP/s", 1e-12),
                    ("update", "k_update (FP64)", "alu", FP64_PEAK_TFLOPS, "TFLOP/s", 1e-12),
                    ("preconditioner", "FP64 AV-MG V-cycle kernels", "hbm", peaks["hbm_gbs"], "GB/s",
                     _vcycle_bytes_per_element(w.mg_levels, 8) * 1e-9)]
    for ph, kernel, bound, peak, unit, per in f64_rows + [
            ("gram_f32", "k_gram_mx (FP32 products, compensated sums)", "alu", fp32_peak, "TFLOP/s", 1e-12),
            ("update_f32", "k_update_mx (FP32 with double-word V part)", "alu", fp32_peak, "TFLOP/s", 1e-12),
            ("preconditioner_f32", "FP32 AV-MG V-cycle kernels", "hbm", peaks["hbm_gbs"], "GB/s",
             _vcycle_bytes_per_element(w.mg_levels, 4) * 1e-9)]:
        d = prof.get(ph)
        if not d or d["ms"] <= 0 or d["work"] <= 0:
            continue
        achieved = d["work"] * per / (d["ms"] / 1e3)
        out.append({"phase": ph, "kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                    "frac": achieved / peak, "total_ms": d["ms"], "calls": d["calls"]})
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
                          switch_tol=args.switch_tol)

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
    with ClockSampler(local) as clk:
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
    roofs = _rooflines(prof, w, peaks, clocks.get("sm_max_mhz"), args.precision == "mixed")
    dom = dict(roofs[0]) if roofs else None
    if dom is not None:
        dom["traffic"] = None
        if dom["phase"] == "gram":
            m_full = 4 * kp
            per = GRAM_DRAM_BYTES_PER_ROW_COL if args.precision == "f64" else GRAM_DW_DRAM_BYTES_PER_ROW_COL
            dom["traffic"] = per * n * m_full
            dom["traffic_note"] = ("ncu dram__bytes_read + write of one %s launch with m = 64 on the 64^3 case, "
                                   "scaled by n m to a 128^3, m = 64 launch (algorithmic bytes 3 n m x 8 = %.3g); "
                                   "%d launches in the timed steps" % (
                                       "k_gram" if args.precision == "f64" else "k_gram_dw", 24.0 * n * m_full,
                                       prof["gram"]["calls"]))
        dom["peak_src"] = ("measured (MEASURED_PEAKS.json hbm_gbs)" if dom["unit"] == "GB/s" else
                           "nominal FP64 rate of the profiling recipe" if "FP64" in dom["kernel"] else
                           "FP32 lanes x clock / 13 x 2 flops (double-word multiply-add = 13 FP32 instructions)" if "double-word" in dom["kernel"]
                           else "FP32 lanes x clock")

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
        "gpu_launches": launches, "roofline": dom, "rooflines": roofs[1:], "clocks": clocks,
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

    w = wl.lap3d_128cube_k10()
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
    with ClockSampler(local) as clk:
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


# Iterations of the FP64 form to relative residual 1e-8 on the 128^3 workload
# (measured on the GPU: 293).  The oracle runs the same FP64 iteration; its
# own count would take over an hour of CPU time to measure.
F64_ITERATIONS_TO_TOL = 293


def run_reference(args, world, rank, local):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.
    Each step times one oracle iteration of the 128^3 workload and scales it
    by the FP64 iteration count to tolerance.  Under torchrun only rank 0
    runs and prints; the other ranks return at once."""
    if rank != 0:
        return
    import workloads as wl
    w = wl.lap3d_128cube_k10()
    iters = F64_ITERATIONS_TO_TOL
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
           "config": lap3d_config(w, "f64", None, "host cores (FP64 oracle)"),
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
    ap.add_argument("--precision", choices=["mixed", "f64"], default="mixed")
    ap.add_argument("--switch-tol", type=float, default=1e-5,
                    help="mixed form: residual level where the FP32 phase hands over to the double-word phase")
    ap.add_argument("--no-f64-compare", action="store_true",
                    help="skip the all-FP64 solve timed beside the mixed-precision steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-grid", type=int, default=0,
                    help="profiling case: N^3 grid of the same problem, fixed iteration count")
    ap.add_argument("--profile-iters", type=int, default=3)
    ap.add_argument("--workload", choices=["lap3d_128cube_k10", "ham64_k8_grad"], default="lap3d_128cube_k10",
                    help="ham64_k8_grad: forward + backward of the 64^3 differentiation workload")
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
        elif args.workload == "ham64_k8_grad":
            run_grad(args, world, rank, local)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1 and args.impl == "ours":
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
