#!/usr/bin/env python
"""Benchmark of multiprecision GMRES on one B300: time to an FP64 relative residual of 1e-10.

A step is one complete GMRES-IR solve (FP32 inner GMRES(50) with FP32 matrix values and FP32
Krylov basis, FP64 residual and update; Algorithm 2) of the 3D 7-point Laplacian 150^3
(n = 3,375,000, nnz = 23,490,000) with b ~ U[-1,1), from x0 = 0.  The same library's FP64
GMRES(50) is timed beside it.  Inputs (FP32 matrix 201 MB, basis 689 MB) are larger than the
126 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With torchrun (N > 1) every rank solves its own system
(independent replicas, weak scaling; the method has no cross-GPU exchange for independent
systems).  ``--impl reference`` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
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
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-10 FP64 residual (s) & solves/s: GMRES-IR FP32 vs FP64 GMRES, 1 B300"
M = 50
TOL = 1e-10
# name -> (generator, polynomial degree, basis precision)
WORKLOADS = {
    "laplace3d_150": ("laplace3d", 0, "f32"),
    "laplace2d_64": ("laplace2d", 0, "f32"),     # the small parity case, latency-bound (in L2)
    "convdiff2d_2500_poly25_bf16": ("convdiff2d", 25, "bf16"),
    "convdiff2d_2500_poly25_f32": ("convdiff2d", 25, "f32"),
    "convdiff2d_2500_poly25_f16": ("convdiff2d", 25, "f16"),
    "batched_256x8_convdiff": ("batched", 0, "bf16"),
    "laplace3d_150_dcgs2": ("laplace3d", 0, "f32"),
    "convdiff2d_2500_poly25_bf16_dcgs2": ("convdiff2d", 25, "bf16"),
}
# workloads run with the delayed-reorthogonalisation variant (gmres_params_t.orth = 1)
ORTH = {"laplace3d_150_dcgs2": 1, "convdiff2d_2500_poly25_bf16_dcgs2": 1}
BATCH_M = 12
WORKLOAD = "laplace3d_150"


def make_workload(name, seed):
    """Matrix, right-hand side and polynomial start vector of a named workload."""
    import synth
    kind, _, _ = WORKLOADS[name]
    if kind == "laplace3d":
        A, b = synth.workload_laplace3d(150, seed)
    elif kind == "laplace2d":
        A, b, _ = synth.workload_laplace2d_64()
    else:
        A, b, _ = synth.workload_convdiff2d(2500, seed)
    return A, b, synth.poly_start_vector(A.n, 0)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 GMRES comparison leg")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-autotune", action="store_true",
                   help="batched workload: keep the default launch shapes")
    p.add_argument("--no-extras", action="store_true",
                   help="default workload: skip the other workloads' keys")
    p.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    p.add_argument("--cpu-reps", type=int, default=1, help=argparse.SUPPRESS)
    p.add_argument("--ncu-batch", action="store_true",
                   help="one directly launched block cycle of the batched workload (for ncu)")
    p.add_argument("--ncu-cycle", choices=["ir", "fp64", "ir-bf16", "ir-dcgs2"],
                   help="run one restart cycle of the workload with direct launches (for ncu)")
    return p.parse_args()


# ------------------------------------------------------------------------------------------
def dist_setup():
    """One process per GPU (torchrun): NCCL when GPUs are present, gloo otherwise (CPU tests)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.seek(0)
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(mhz)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# The files that define the single-system kernels and their launch shapes: a DRAM-traffic figure
# taken with ncu stays valid while these are unchanged.
KERNEL_SOURCES = ("common.cuh", "kernels.cuh", "cluster_cycle.cuh", "solver.cu")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2105_07544_b300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on these sources."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    if not m or m.group(1) != kernel_source_hash():
        return None
    m = re.search(rf"^\|\s*{kernel_class}\s*\|\s*([0-9.eE+]+)\s*\|", text, re.M)
    return float(m.group(1)) if m else None


# ------------------------------------------------------------------------------------------
THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
              "NUMEXPR_NUM_THREADS", "VECLIB_MAXIMUM_THREADS")

# With a polynomial, one oracle cycle of 50 steps takes minutes on one core; the sample is the
# first steps of a cycle, extrapolated linearly by iterations (the polynomial's SpMVs dominate).
POLY_SAMPLE_STEPS = 4


def _cpu_sample_main(workload, reps):
    """Child process (BLAS/OpenMP threads set through the environment): time `reps` bounded
    samples of the oracle on the workload and print them as one JSON line.  Single-system
    workloads: one FP32-inner GMRES(50) cycle (with the workload's polynomial and basis rounding)
    plus its FP64 residual, or with a polynomial the first POLY_SAMPLE_STEPS steps of that cycle.
    Batched: the whole block GMRES-IR solve of system 1 (8 right-hand sides).  The inputs are
    built once, outside the timed samples."""
    import synth
    from oracle import gmres as og
    times = []
    if WORKLOADS[workload][0] == "batched":
        from oracle import block
        A, B = synth.workload_batched()[1]
        for _ in range(reps):
            t0 = time.perf_counter()
            block.block_gmres_ir(A, B, BATCH_M, TOL, basis="bf16")
            times.append(time.perf_counter() - t0)
        print(json.dumps({"seconds": times, "n": A.n, "columns": B.shape[1]}), flush=True)
        return
    A, b, pstart = make_workload(workload, 0)
    _, degree, basis = WORKLOADS[workload]
    poly = og.poly_build(A, degree, pstart) if degree > 0 else None   # untimed, as on the GPU
    steps = M if poly is None else POLY_SAMPLE_STEPS
    rnd = {"bf16": og.round_bf16, "f16": og.round_f16_scaled}.get(basis)
    cycle = og.gmres_cycle_dcgs2 if ORTH.get(workload, 0) else og.gmres_cycle
    for _ in range(reps):
        t0 = time.perf_counter()
        r = b - og.spmv(A, np.zeros(A.n))
        if poly is None:
            op = lambda z: og.spmv(A, z, np.float32)
        else:
            op = lambda z: og.spmv(A, og.poly_apply(A, poly, z, np.float32), np.float32)
        cyc = cycle(op, r.astype(np.float32), steps, dtype=np.float32, basis_round=rnd)
        u = cyc.V[:, : cyc.k] @ cyc.y.astype(np.float32)
        if poly is not None:
            u = og.poly_apply(A, poly, u, np.float32)
        _ = b - og.spmv(A, u.astype(np.float64))
        times.append(time.perf_counter() - t0)
    print(json.dumps({"seconds": times, "steps": steps}), flush=True)


def cpu_oracle_samples(workload, threads, reps=1):
    """Run `reps` oracle samples of the workload in one child process with `threads` BLAS and
    OpenMP threads; returns its JSON (per-sample seconds)."""
    env = dict(os.environ)
    for k in THREAD_ENV:
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", workload,
                          "--cpu-reps", str(reps)],
                         env=env, capture_output=True, text=True, check=True).stdout
    return json.loads(out.strip().splitlines()[-1])


def oracle_cycles_needed(workload):
    """Restart cycles the oracle's own GMRES-IR needs on the workload (its golden run), if known."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_laplace3d_150.json")
    if workload == WORKLOAD and os.path.exists(path):
        return int(json.load(open(path))["ir"]["cycles"]), "the oracle's golden run"
    return None, None


# GPU iteration and cycle counts of the single-system workloads (tol 1e-10, GMRES(50), seed 0),
# used to extrapolate the oracle's bounded samples to a whole solve when the oracle's own count
# is not stored.
GPU_COUNTS = {"laplace3d_150": (1550, 31), "laplace3d_150_dcgs2": (1550, 31),
              "laplace2d_64": (350, 7), "convdiff2d_2500_poly25_bf16": (750, 15),
              "convdiff2d_2500_poly25_f32": (800, 16), "convdiff2d_2500_poly25_f16": (800, 16),
              "convdiff2d_2500_poly25_bf16_dcgs2": (800, 16)}


def oracle_rate(workload, sample_s, steps, gpu_iters, gpu_cycles):
    """(value, unit, extrapolation dict) of the oracle from one sample's seconds."""
    if WORKLOADS[workload][0] == "batched":
        return 8.0 / sample_s, "column solves/s", {
            "factor": 1, "sampled": "the whole block GMRES-IR solve of system 1 (8 columns)",
            "to": "column solves/s of that system"}
    if steps == M:
        cycles, src = oracle_cycles_needed(workload)
        if cycles is None:
            cycles, src = gpu_cycles, "the GPU's cycle count for this workload"
        return 1.0 / (sample_s * cycles), "solves/s", {
            "factor": cycles, "sampled": f"one GMRES-IR cycle ({M} FP32 Arnoldi steps + FP64 "
            f"residual)", "to": f"one solve = {cycles} cycles ({src})"}
    return 1.0 / (sample_s / steps * gpu_iters), "solves/s", {
        "factor": gpu_iters / steps, "sampled": f"the first {steps} steps of a GMRES-IR cycle "
        "(polynomial applied per step)", "to": f"one solve = {gpu_iters} iterations (the GPU's "
        "count), linearly"}


def cpu_baseline_of(workload, gpu_iters, gpu_cycles):
    """cpu_baseline of the line: the oracle on one host thread and on all of them."""
    cores = os.cpu_count() or 1
    d1 = cpu_oracle_samples(workload, 1)
    v1, unit, ext = oracle_rate(workload, d1["seconds"][0], d1.get("steps", M), gpu_iters,
                                gpu_cycles)
    dn = cpu_oracle_samples(workload, cores)
    vn, _, _ = oracle_rate(workload, dn["seconds"][0], dn.get("steps", M), gpu_iters, gpu_cycles)
    return {"value": v1, "unit": unit, "cores": 1, "kind": "oracle",
            "sample": f"{ext['sampled']}: {d1['seconds'][0]:.2f} s on 1 thread, "
                      f"{dn['seconds'][0]:.2f} s on {cores}; extrapolated to {ext['to']}",
            "extrapolation": ext,
            "all_cores": {"value": vn, "unit": unit, "cores": cores,
                          "sample_s": dn["seconds"][0]}}


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle, as it stands, on all host cores.  Every step (warm-up
    included) is one bounded sample of the workload (one GMRES-IR cycle; the first steps of a
    cycle with a polynomial; one system's block solve when batched), all in one child process;
    ms_per_step is the measured time of a sample, value the workload's metric extrapolated from
    the median sample (the factor is in `extrapolation`)."""
    if rank != 0:
        return
    iters, cycles = GPU_COUNTS.get(args.workload, (0, 0))
    cores = os.cpu_count() or 1
    d = cpu_oracle_samples(args.workload, cores, args.warmup + args.steps)
    samples = d["seconds"][args.warmup:]
    med = statistics.median(samples)
    value, unit, ext = oracle_rate(args.workload, med, d.get("steps", M), iters, cycles)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": med * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 inner / f64 outer", "data": "synthetic",
            "config": {"workload": args.workload, "m": BATCH_M if unit == "column solves/s" else M,
                       "tol": TOL, "rhs": "uniform[-1,1) seed 0"},
            "extrapolation": ext,
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": f"{ext['sampled']} per step, median {med:.2f} s; "
                                       f"extrapolated to {ext['to']}"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
def time_calls(fn, steps, warmup):
    """Seconds per call of fn() (a whole solve returning stats) by CUDA events on the current
    stream, after `warmup` untimed calls; returns (seconds, last stats, kernel launches)."""
    import torch
    for _ in range(warmup):
        st = fn()
        assert st.converged, st
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(stream)
    for _ in range(steps):
        st = fn()
        launches += st.kernel_launches
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3 / steps, st, launches


def measure_batched(rank, steps, warmup, autotune=True, profile=True):
    """The batched workload (256 uneven convection-diffusion systems x 8 right-hand sides, block
    GMRES-IR with tensor-core block CGS2, one graph per block cycle): per-solve time by CUDA
    events, end-to-end time with host buffers, and the block-sweep roofline of one profiled
    block cycle."""
    import torch

    import paper_2105_07544_b300 as g
    import synth
    from paper_2105_07544_b300 import roofline

    wl = synth.workload_batched(seed0=1000 * rank)
    bs = g.BatchSolver([A for A, _ in wl], m=BATCH_M)
    Bflat = torch.from_numpy(bs.pack([B for _, B in wl])).cuda()
    ncol = len(wl) * 8
    X = torch.zeros_like(Bflat)
    tuned = None
    if autotune:   # launch shapes: the tuning cache, else the autotuner (untimed)
        from paper_2105_07544_b300 import autotune as at
        tuned = at.tune_batch(bs, Bflat, sum(A.nnz for A, _ in wl), BATCH_M, tol=TOL)
        tuned = {"shapes": tuned["shapes"], "cached": tuned["cached"],
                 "solve_s": round(tuned["s_per_iter"], 4),
                 "default_solve_s": round(tuned["default_s_per_iter"], 4)}

    def solve():
        X.zero_()
        return bs.ir_solve(Bflat, X, tol=TOL)[1]

    t_step, st, launches = time_calls(solve, steps, warmup)
    # end to end with host buffers (pinned), copies inside the timed region
    bh = torch.from_numpy(bs.pack([B for _, B in wl])).pin_memory().numpy()
    xh = torch.zeros(bh.shape[0], dtype=torch.float64).pin_memory().numpy()
    t0 = time.perf_counter()
    for _ in range(steps):
        xh[:] = 0.0
        bs.ir_solve(bh, xh, tol=TOL)
    t_e2e = (time.perf_counter() - t0) / steps
    roof = None
    if profile:
        # roofline of the dominant kernel class (the block-CGS2 sweeps): one block cycle with
        # every system active, kernel classes timed with CUDA events on the batch's stream
        bs.set_profiling(True)
        X.zero_()
        _, sp = bs.ir_solve(Bflat, X, tol=TOL, max_cycles=1)
        bs.set_profiling(False)
        n_pad = sum(-(-A.n // 128) * 128 for A, _ in wl)
        sweep_bytes = roofline.batch_sweep_bytes(n_pad, BATCH_M)
        nl = max(1, sp.class_launches["sweep"])
        peak, peak_kind = measured_peak()
        achieved = sweep_bytes / sp.t_kernel["sweep"] / 1e9
        roof = {"bound": "hbm", "kernel": "kb_sweep (block CGS2, tensor cores)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind, "traffic": None,
                "algorithmic_bytes_per_launch": sweep_bytes / nl,
                "avg_launch_ms": sp.t_kernel["sweep"] / nl * 1e3,
                "per_class_s": {k: round(v, 6) for k, v in sp.t_kernel.items()},
                "measured_in": "the first block cycle (all systems active) of one extra solve "
                               "with per-class CUDA events on the batch's stream (direct launches)"}
    out = {"column_solves_per_s": ncol / t_step, "time_to_solution_s": t_step,
           "systems": len(wl), "nrhs": 8, "rows": sum(A.n for A, _ in wl),
           "nnz": sum(A.nnz for A, _ in wl), "block_steps_per_cycle": BATCH_M,
           "cycles": st.cycles, "block_steps_total": st.block_steps,
           "max_rel_res": st.max_rel_res, "converged_systems": st.converged_systems,
           "launch_shapes": tuned, "e2e_column_solves_per_s": ncol / t_e2e,
           "h2d_bytes_per_step": 2 * 8 * bh.shape[0], "d2h_bytes_per_step": 8 * bh.shape[0],
           "gpu_launches": launches, "roofline": roof}
    bs.close()
    return out


def run_batched(args, world, rank):
    """The batched workload as the line's own metric (column solves per second)."""
    barrier(world)
    import torch
    with Clocks(torch.cuda.current_device()) as clk:
        r = measure_batched(rank, args.steps, args.warmup, autotune=not args.no_autotune)
    t_step = max_over_ranks(r["time_to_solution_s"], world)
    if rank == 0:
        cpu = cpu_baseline_of(args.workload, 0, 0) if world == 1 and not args.no_cpu else None
        line = {"metric": METRIC, "value": world * r["systems"] * 8 / t_step,
                "unit": "column solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_step * 1e3, "time_to_solution_s": t_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16 basis / f32 inner / f64 outer", "data": "synthetic",
                "config": {"workload": args.workload, "systems": r["systems"], "nrhs": 8,
                           "rows": r["rows"], "nnz": r["nnz"], "block_steps": BATCH_M,
                           "tol": TOL, "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2 (126 MB); no flush",
                           "launch_shapes": r["launch_shapes"]},
                "cycles": r["cycles"], "block_steps_total": r["block_steps_total"],
                "max_rel_res": r["max_rel_res"], "converged_systems": r["converged_systems"],
                "e2e": {"value": world * r["e2e_column_solves_per_s"], "unit": "column solves/s",
                        "h2d_bytes_per_step": r["h2d_bytes_per_step"],
                        "d2h_bytes_per_step": r["d2h_bytes_per_step"]},
                "gpu_launches": r["gpu_launches"], "clocks": clk.summary(),
                "roofline": r["roofline"], "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)


def solution_error(x):
    """Relative error of the 150^3 GMRES-IR solution (seed-0 right-hand side) at the oracle's 64
    sampled rows: against the oracle's GMRES-IR runs to 1e-12 and to 1e-10 (tests/golden, written
    by scripts that call only the oracle), with the bound kappa(A) * 1e-10 of a 1e-10 residual
    (kappa of the 3D Laplacian from its closed-form extreme eigenvalues)."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_laplace3d_150.json")
    if not os.path.exists(path):
        return None
    gold = json.load(open(path))
    rows = np.array(gold["sample_rows"])
    xs = x.cpu().numpy()[rows]
    out = {"rows": len(rows)}
    for key, name in (("ir_tol1e-12", "vs_oracle_ir_tol1e-12"), ("ir", "vs_oracle_ir_tol1e-10")):
        if key in gold:
            xo = np.array(gold[key]["x_sample"])
            out[name] = float(np.linalg.norm(xs - xo) / np.linalg.norm(xo))
    N = 150
    lmin = 3 * (2 - 2 * np.cos(np.pi / (N + 1)))
    lmax = 3 * (2 - 2 * np.cos(N * np.pi / (N + 1)))
    out["bound_kappa_x_1e-10"] = lmax / lmin * TOL
    return out


def measure_extras(steps, warmup):
    """The other workloads of the benchmark, timed the same way (CUDA events around whole
    solves, inputs resident, nothing skipped): the delayed-reorthogonalisation variant on
    150^3, the 2500^2 convection-diffusion problem with the degree-25 polynomial (GMRES-IR with
    BF16 and FP32 bases, and FP64 GMRES), and the batched workload."""
    import torch

    import paper_2105_07544_b300 as g

    extras = {}
    k, w = max(1, min(steps, 3)), 1
    # 2500^2 convection-diffusion, degree-25 polynomial
    A, b, pstart = make_workload("convdiff2d_2500_poly25_bf16", 0)
    bd = torch.from_numpy(b).cuda()
    c3 = {"n": A.n, "nnz": A.nnz, "poly_degree": 25, "m": M, "tol": TOL}
    for basis in ("bf16", "f32"):
        s = g.Solver(A, m=M, poly_degree=25, basis=basis, poly_start=pstart)
        x = torch.zeros_like(bd)

        def ir():
            x.zero_()
            return s.ir_solve(bd, x, tol=TOL)[1]

        t, st, _ = time_calls(ir, k, w)
        c3[f"ir_{basis}"] = {"time_to_solution_s": t, "iters": st.iters, "cycles": st.cycles,
                             "rel_res": st.rel_res}
        if basis == "f32":
            def f64():
                x.zero_()
                return s.solve_fp64(bd, x, tol=TOL)[1]

            t, st, _ = time_calls(f64, max(1, min(steps, 2)), w)
            c3["fp64_gmres"] = {"time_to_solution_s": t, "iters": st.iters, "rel_res": st.rel_res}
        s.close()
    c3["speedup_ir_bf16_over_fp64"] = c3["fp64_gmres"]["time_to_solution_s"] / \
        c3["ir_bf16"]["time_to_solution_s"]
    extras["convdiff2d_2500_poly25"] = c3
    # batched
    r = measure_batched(0, max(1, min(steps, 5)), w, autotune=True, profile=True)
    extras["batched_256x8_convdiff"] = {k2: r[k2] for k2 in (
        "column_solves_per_s", "time_to_solution_s", "e2e_column_solves_per_s", "cycles",
        "block_steps_total", "max_rel_res", "converged_systems", "systems", "rows", "nnz",
        "launch_shapes")}
    extras["batched_256x8_convdiff"]["roofline_frac_block_sweeps"] = \
        r["roofline"]["frac"] if r["roofline"] else None
    return extras


def run_ours(args, world, rank):
    import torch

    import paper_2105_07544_b300 as g
    from paper_2105_07544_b300 import roofline

    A, b, pstart = make_workload(args.workload, rank)   # each rank: its own right-hand side
    _, degree, basis = WORKLOADS[args.workload]
    orth = ORTH.get(args.workload, 0)
    s = g.Solver(A, m=M, poly_degree=degree, basis=basis, poly_start=pstart)
    s.set_params(orth=orth)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)

    def solve_ir():
        x.zero_()
        return s.ir_solve(bd, x, tol=TOL)[1]

    for _ in range(args.warmup):
        st = solve_ir()
        assert st.converged, st
    torch.cuda.synchronize()
    barrier(world)
    launches = 0
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        stats = []
        for _ in range(args.steps):
            st = solve_ir()
            stats.append(st)
            launches += st.kernel_launches
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    elapsed = max_over_ranks(e0.elapsed_time(e1) * 1e-3, world)
    t_step = elapsed / args.steps
    value = world / t_step
    st = stats[-1]
    # independent check of the returned x: FP64 residual through the library's FP64 SpMV
    resid = float(torch.linalg.norm(bd - s.spmv(x, "f64")) / torch.linalg.norm(bd))
    err = solution_error(x) if args.workload in (WORKLOAD, "laplace3d_150_dcgs2") and rank == 0 \
        else None

    # FP64 GMRES leg (the comparison the metric names), with the paper's CGS2
    fp64 = None
    if not args.no_fp64:
        s.set_params(orth=0)

        def solve_f64():
            x.zero_()
            return s.solve_fp64(bd, x, tol=TOL)[1]

        tf, sf, _ = time_calls(solve_f64, max(1, min(args.steps, 2)), 1)
        fp64 = {"time_to_solution_s": tf, "iters": sf.iters, "converged": sf.converged,
                "rel_res": sf.rel_res, "speedup_ir_over_fp64": tf / t_step}
        s.set_params(orth=orth)

    # the delayed-reorthogonalisation variant of the same solve (a different algorithm)
    dcgs2 = None
    if args.workload == WORKLOAD:
        s.set_params(orth=1)
        td, sd, _ = time_calls(solve_ir, max(1, min(args.steps, 5)), 2)
        dcgs2 = {"time_to_solution_s": td, "iters": sd.iters, "cycles": sd.cycles,
                 "rel_res": sd.rel_res, "speedup_over_cgs2": t_step / td}
        s.set_params(orth=orth)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros(A.n, dtype=torch.float64).pin_memory()
    bnp, xnp = bh.numpy(), xh.numpy()
    s.ir_solve(bnp, xnp, tol=TOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xnp[:] = 0.0
        _, se = s.ir_solve(bnp, xnp, tol=TOL)
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / args.steps
    e2e = {"value": world / max_over_ranks(t_e2e, world), "unit": "solves/s",
           "h2d_bytes_per_step": 2 * 8 * A.n, "d2h_bytes_per_step": 8 * A.n}

    # per-kernel-class event timing of one more solve of the same workload (profiling mode)
    s.set_params(profiling=1)
    x.zero_()
    _, sp = s.ir_solve(bd, x, tol=TOL)
    s.set_params(profiling=0)
    sv = 2 if basis == "bf16" else 4
    byts = (roofline.dcgs2_cycle_bytes(A.n, A.nnz, M, 4, sv, 4) if orth else
            roofline.cycle_bytes(A.n, A.nnz, M, 4, sv, 4))    # per cycle, per class
    per_cycle = {k: (1 if k == "cgs_proj" else M) for k in byts}   # launches per cycle
    if degree > 0:
        byts["precond"] = degree * M * roofline.poly_step_bytes(A.n, A.nnz)
        per_cycle["precond"] = degree * M
    timed = {k: sp.t_kernel[k] for k in byts if sp.t_kernel.get(k, 0) > 0}
    dom = max(timed, key=timed.get)
    avg_dur = sp.t_kernel[dom] / (per_cycle[dom] * sp.cycles)
    alg_bytes = byts[dom] / per_cycle[dom]
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / avg_dur / 1e9
    traffic = ncu_traffic(dom) if args.workload == WORKLOAD else None
    names = {"spmv": "k_spmv_proj (inner SpMV fused with the first CGS2 projection)",
             "cgs_pass2": "k_sweep<PASS2>", "cgs_update": "k_sweep<UPDATE>",
             "precond": "k_poly_step (polynomial SpMV step)"}
    if orth:
        names.update({"spmv": "k_dc_reduce (SpMV fused with the DCGS2 reduction)",
                      "cgs_update": "k_sweep<DC_UPDATE>"})
    roof = {"bound": "hbm", "kernel": names.get(dom, dom), "class": dom, "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
            "traffic": traffic, "algorithmic_bytes_per_launch": alg_bytes,
            "avg_launch_ms": avg_dur * 1e3,
            "per_class_s": {k: round(v, 5) for k, v in sp.t_kernel.items() if v > 0},
            "per_class_frac_of_hbm": {
                k: (byts[k] / per_cycle[k]) / (sp.t_kernel[k] / (per_cycle[k] * sp.cycles)) / 1e9 / peak
                for k in timed},
            "measured_in": "one extra solve of the same workload with per-class CUDA events on "
                           "the library stream (profiling mode, no graph)"}
    if st.kernel_launches <= st.cycles + 2:
        # the timed solves ran each cycle as one kernel on one thread-block cluster (a small
        # system); the profiling-mode classes above are those of the per-step kernels
        cyc_bytes = sum(byts[k] for k in byts if k != "precond")
        t_cycle = t_step / max(1, st.cycles)
        achieved_c = cyc_bytes / t_cycle / 1e9
        roof = {"bound": "hbm", "kernel": "k_cycle_cluster (one restart cycle on one thread-block "
                "cluster)", "class": "cycle", "achieved": achieved_c, "peak": peak, "unit": "GB/s",
                "frac": achieved_c / peak, "peak_kind": peak_kind, "traffic": None,
                "algorithmic_bytes_per_launch": cyc_bytes, "avg_launch_ms": t_cycle * 1e3,
                "note": "latency-bound: the whole system sits in the cluster's shared memory; "
                        "dependent FP64 operations and three cluster barriers per step set the time",
                "per_step_kernels_profiled": roof}

    extras = None
    if world == 1 and rank == 0 and args.workload == WORKLOAD and not args.no_extras:
        s.close()
        s = None
        extras = measure_extras(args.steps, args.warmup)
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu:
            cpu = cpu_baseline_of(args.workload, st.iters, st.cycles)
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
                "time_to_solution_s": t_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 inner / f64 outer", "data": "synthetic",
                "config": {"workload": args.workload, "n": A.n, "nnz": A.nnz, "m": M, "tol": TOL,
                           "inner": "f32", "basis": basis, "matrix": "f32 copy of f64",
                           "poly_degree": degree,
                           "orthogonalisation": "dcgs2" if orth else "cgs2",
                           "rhs": ("A x*, x* uniform[0,1) seed 0" if WORKLOADS[args.workload][0] == "laplace2d"
                                   else "uniform[-1,1) seed = rank"),
                           "parallelism": f"replicas x{world}",
                           "l2": ("inputs larger than L2 (126 MB); no flush"
                                  if A.nnz * 12 + A.n * 8 * (M + 4) > 126e6 else
                                  "the whole problem fits in L2 (latency-bound case); no flush")},
                "iters": st.iters, "cycles": st.cycles, "rel_res": st.rel_res,
                "rel_res_check": resid, "solution_error": err, "fp64_gmres": fp64,
                "dcgs2": dcgs2, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
                "roofline": roof, "cpu_baseline": cpu, "workloads": extras}
        print(json.dumps(line), flush=True)
    if s is not None:
        s.close()


def run_ncu_batch():
    """One block cycle of the batched workload, kernels launched directly (profiling mode), so
    that a profiler sees each launch: per block step k an SpMM, the three block-CGS2 sweeps
    (kb_sweep) and the per-system small kernels."""
    import torch

    import paper_2105_07544_b300 as g
    import synth
    torch.cuda.set_device(0)
    wl = synth.workload_batched()
    bs = g.BatchSolver([A for A, _ in wl], m=BATCH_M)
    B = torch.from_numpy(bs.pack([B for _, B in wl])).cuda()
    bs.set_profiling(True)
    _, st = bs.ir_solve(B, tol=TOL, max_cycles=1)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_batch": True, "cycles": st.cycles, "launches": st.kernel_launches,
                      "n_padded": sum(-(-A.n // 128) * 128 for A, _ in wl)}))
    bs.close()


def run_ncu_cycle(kind, workload=WORKLOAD):
    """One 50-step restart cycle of a single-system workload, kernels launched directly (no
    graph), so that a profiler sees each launch: 1 norm + 1 residual + 50 steps (FP32: the SpMV
    fused with the first projection and two CGS2 sweeps; FP64: the SpMV and three sweeps; with a
    polynomial, its SpMV steps first) + the cycle-end kernels."""
    import torch

    import paper_2105_07544_b300 as g
    torch.cuda.set_device(0)
    A, b, pstart = make_workload(workload, 0)
    _, degree, _ = WORKLOADS[workload]
    s = g.Solver(A, m=M, poly_degree=degree, poly_start=pstart,
                 basis="bf16" if kind == "ir-bf16" else "f32")
    s.set_params(use_graphs=0, maxiter=M, orth=1 if kind == "ir-dcgs2" else 0)
    bd = torch.from_numpy(b).cuda()
    _, st = (s.solve_fp64 if kind == "fp64" else s.ir_solve)(bd, tol=TOL)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_cycle": kind, "iters": st.iters, "launches": st.kernel_launches}))


def main():
    args = parse()
    if args.cpu_sample:
        _cpu_sample_main(args.cpu_sample, args.cpu_reps)
        return
    if args.ncu_cycle:
        run_ncu_cycle(args.ncu_cycle, args.workload)
        return
    if args.ncu_batch:
        run_ncu_batch()
        return
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, world, rank)
        return
    world, rank = dist_setup()
    if WORKLOADS[args.workload][0] == "batched":
        run_batched(args, world, rank)
    else:
        run_ours(args, world, rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
