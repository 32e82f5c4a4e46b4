"""Experiment drivers for the paper's precision studies (run on the GPU).

``bjacobi``: block Jacobi after RCM reordering (Section V-G's recipe; its SuiteSparse matrices
are not available, so a randomly relabelled heterogeneous-coefficient 2D diffusion problem
stands in: row scales spread over four orders of magnitude, and the relabelling destroys the
natural ordering, which RCM restores).  Block sizes 1 and 42, solved with
FP64 GMRES (FP64 blocks, and FP32 blocks: variant (a) of Section III-D) and GMRES-IR (FP32
blocks: variant (b)), beside the unpreconditioned solves.

``fd``: GMRES-FD against GMRES-IR and FP64 GMRES (Section V-A).  GMRES-FD runs single-precision
GMRES(50) up to a switch point and FP64 GMRES(50) from its iterate; the study sweeps the switch
point over restarts and records total iterations and time beside one GMRES-IR and one FP64 run
(b = ones, x0 = 0, tol 1e-10).

``loa``: the loss-of-accuracy study of Section V-F.  A 3D Laplacian (200 points per direction by
default, b = ones, x0 = 0, GMRES(50), tol 1e-10) is polynomial-preconditioned with degrees
10, 20, ..., 70 and solved three ways: FP64 GMRES with the polynomial applied in FP64, FP64 GMRES
with the polynomial applied in FP32 (variant (a) of Section III-D), and GMRES-IR (FP32 inner
cycle and polynomial, FP64 residual).  For each it records convergence, iterations, restarts,
loss-of-accuracy events (the implicit residual met the tolerance, the explicit one did not) and
the solve time.  This library's FP64 solver restarts from the explicit residual after such an
event instead of stopping, which is the correction the paper suggests.
"""
from __future__ import annotations

import json
import time

import numpy as np


def _solve(s, fn, bd, tol):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, st = fn(bd, tol=tol)
    torch.cuda.synchronize()
    return dict(converged=bool(st.converged), iters=int(st.iters), cycles=int(st.cycles),
                rel_res=float(st.rel_res), loss_of_accuracy=int(st.loss_of_accuracy),
                seconds=time.perf_counter() - t0)


def loa(N=200, degrees=(10, 20, 30, 40, 50, 60, 70), m=50, tol=1e-10, max_loa=20, log=print):
    import torch
    import synth
    from . import Solver
    A = synth.laplace3d(N)
    bd = torch.ones(A.n, dtype=torch.float64, device="cuda")
    start = synth.poly_start_vector(A.n)
    rows = []
    for d in degrees:
        row = dict(degree=d)
        for name, prec in (("fp64_poly64", "f64"), ("fp64_poly32", "f32")):
            s = Solver(A, m=m, poly_degree=d, poly_start=start, fp64_precond=prec)
            s.set_params(max_loss_of_accuracy=max_loa)
            s.solve_fp64(bd, tol=tol)                   # warm-up (graph capture)
            row[name] = _solve(s, s.solve_fp64, bd, tol)
            if prec == "f32":
                s.ir_solve(bd, tol=tol)
                row["ir_poly32"] = _solve(s, s.ir_solve, bd, tol)
            s.close()
        rows.append(row)
        log(json.dumps(row), flush=True)
    return rows


def fd(problem="laplace3d_200", switches=None, m=50, tol=1e-10, log=print):
    import torch
    import synth
    from . import Solver
    if problem == "laplace3d_200":
        A = synth.laplace3d(200)
    elif problem == "convdiff2d_2500":
        A, _, _ = synth.workload_convdiff2d(2500, 0)
    else:
        raise ValueError(problem)
    bd = torch.ones(A.n, dtype=torch.float64, device="cuda")
    s = Solver(A, m=m)
    s.set_params(max_loss_of_accuracy=1 << 30)
    out = dict(problem=problem, n=A.n)
    s.ir_solve(bd, tol=tol)                          # warm-ups (graph capture)
    out["ir"] = _solve(s, s.ir_solve, bd, tol)
    s.solve_fp64(bd, tol=tol)
    out["fp64"] = _solve(s, s.solve_fp64, bd, tol)
    log(json.dumps(out), flush=True)
    if switches is None:
        top = out["ir"]["iters"]
        step = max(m, (top // 10) // m * m)
        switches = list(range(step, top + step, step))
    rows = []
    for sw in switches:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, st, k = s.fd_solve(bd, sw, tol=tol)
        torch.cuda.synchronize()
        row = dict(switch=sw, fp32_iters=int(k), iters=int(st.iters), converged=bool(st.converged),
                   rel_res=float(st.rel_res), seconds=time.perf_counter() - t0)
        rows.append(row)
        log(json.dumps(row), flush=True)
    s.close()
    out["fd"] = rows
    return out


def bjacobi(N=400, contrast=1e4, blocks=(0, 1, 42), m=50, tol=1e-10, log=print):
    import torch
    import synth
    from . import Solver
    A = synth.permute_symmetric(synth.hetero2d(N, contrast, 0), 1)
    b = synth.uniform(A.n, 0)
    bd = torch.from_numpy(b).cuda()
    rows = []
    for k in blocks:
        row = dict(block=k, n=A.n)
        for name, prec, fn in (("fp64", "f64", "solve_fp64"), ("fp64_bj32", "f32", "solve_fp64"),
                               ("ir", "f64", "ir_solve")):
            if k == 0 and name == "fp64_bj32":
                continue
            s = Solver(A, m=m, fp64_precond=prec)
            t0 = time.perf_counter()
            if k:
                s.set_block_jacobi(k, reorder=True)
            row[f"setup_s_{name}"] = time.perf_counter() - t0
            s.set_params(max_loss_of_accuracy=1 << 30, maxiter=100000)
            f = getattr(s, fn)
            f(bd, tol=tol)                              # warm-up (graph capture)
            row[name] = _solve(s, f, bd, tol)
            s.close()
        rows.append(row)
        log(json.dumps(row), flush=True)
    return rows


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="precision studies of the paper")
    ap.add_argument("study", choices=["loa", "fd", "bjacobi"])
    ap.add_argument("--N", type=int, default=200)
    ap.add_argument("--degrees", default="10,20,30,40,50,60,70")
    ap.add_argument("--problem", default="laplace3d_200")
    ap.add_argument("--out")
    a = ap.parse_args(argv)
    if a.study == "loa":
        rows = loa(a.N, tuple(int(v) for v in a.degrees.split(",")))
    elif a.study == "bjacobi":
        rows = bjacobi()
    else:
        rows = fd(a.problem)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
