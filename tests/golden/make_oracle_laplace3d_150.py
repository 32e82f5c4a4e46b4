"""Write oracle_laplace3d_150.json: the CPU oracle's GMRES-IR and FP64 GMRES(50) runs on the
3D 7-point Laplacian 150^3 with b ~ U[-1,1) seed 0, tol 1e-10 (calls only oracle/ and synth/).

Stored: iteration and cycle counts, final explicit residuals, per-cycle residual history and
x at 64 seeded sample rows, used by the full-size GPU parity test.  Takes tens of minutes.

    python tests/golden/make_oracle_laplace3d_150.py          # the tol 1e-10 runs
    python tests/golden/make_oracle_laplace3d_150.py --tight  # add GMRES-IR to tol 1e-12

The tight run's x (same sample rows) is the reference the benchmark measures the solution error
of its 1e-10 solves against.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import gmres as og  # noqa: E402


def tight():
    path = os.path.join(HERE, "oracle_laplace3d_150.json")
    out = json.load(open(path))
    A, b = synth.workload_laplace3d(150, 0)
    rows = np.array(out["sample_rows"])
    t = time.time()
    ir = og.gmres_ir(A, b, m=50, tol=1e-12)
    out["ir_tol1e-12"] = {"iters": ir.iters, "cycles": ir.cycles, "rel_res": ir.rel_res,
                          "x_sample": ir.x[rows].tolist(), "seconds": time.time() - t}
    print("ir 1e-12", ir.iters, ir.cycles, ir.rel_res, time.time() - t, flush=True)
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)


def main():
    A, b = synth.workload_laplace3d(150, 0)
    rows = np.sort(np.random.default_rng(123).choice(A.n, 64, replace=False))
    out = {"_source": "tests/golden/make_oracle_laplace3d_150.py (oracle only)",
           "workload": "laplace3d_150, b ~ U[-1,1) seed 0, m = 50, tol 1e-10",
           "sample_rows": rows.tolist()}
    t = time.time()
    ir = og.gmres_ir(A, b, m=50, tol=1e-10)
    out["ir"] = {"iters": ir.iters, "cycles": ir.cycles, "rel_res": ir.rel_res,
                 "history": ir.history, "x_sample": ir.x[rows].tolist(),
                 "seconds": time.time() - t}
    print("ir", ir.iters, ir.cycles, ir.rel_res, time.time() - t, flush=True)
    t = time.time()
    f = og.gmres(A, b, m=50, tol=1e-10)
    out["fp64"] = {"iters": f.iters, "cycles": f.cycles, "rel_res": f.rel_res,
                   "history": f.history, "x_sample": f.x[rows].tolist(),
                   "seconds": time.time() - t}
    print("fp64", f.iters, f.cycles, f.rel_res, time.time() - t, flush=True)
    with open(os.path.join(HERE, "oracle_laplace3d_150.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    tight() if "--tight" in sys.argv else main()
