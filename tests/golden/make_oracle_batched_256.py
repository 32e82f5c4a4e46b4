"""Write oracle_batched_256.json: the CPU oracle's block GMRES-IR on a sample of the batched
workload (256 convection-diffusion systems, sides U{32..320}, diagonal shift U[0, 0.5], Peclet
100, 8 right-hand sides U[-1,1) each; system s from default_rng(s)), restart 12 block steps,
BF16 basis, tol 1e-10.  Calls only oracle/ and synth/.

Sample: the three largest systems, the two smallest and three more drawn with default_rng(7).
Stored per system: block cycles, per-column final relative residuals, and at 16 seeded rows the
block GMRES-IR solution and the FP64 GMRES(60) solution of each column to tol 1e-13 (the sharp
reference the GPU solution is compared with).  Takes a few minutes.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import block as ob  # noqa: E402
from oracle import gmres as og  # noqa: E402

M, TOL = 12, 1e-10


def sample_indices(wl):
    n = np.array([A.n for A, _ in wl])
    order = np.argsort(n, kind="stable")
    pick = list(order[-3:]) + list(order[:2])
    rest = [i for i in range(len(wl)) if i not in pick]
    pick += list(np.random.default_rng(7).choice(rest, 3, replace=False))
    return sorted(int(i) for i in pick)


def main():
    wl = synth.workload_batched()
    out = {"_source": "tests/golden/make_oracle_batched_256.py (oracle only)",
           "workload": "batched_256x8_convdiff (seed0 0), block GMRES-IR, m = 12 block steps, "
                       "bf16 basis, tol 1e-10", "systems": []}
    for s in sample_indices(wl):
        A, B = wl[s]
        rows = np.sort(np.random.default_rng(100 + s).choice(A.n, 16, replace=False))
        t = time.time()
        r = ob.block_gmres_ir(A, B, M, TOL, basis="bf16", maxcycles=2000)
        t_ir = time.time() - t
        X64 = np.column_stack([og.gmres(A, B[:, c], 60, 1e-13).x for c in range(B.shape[1])])
        out["systems"].append({"index": s, "n": A.n, "cycles": r.cycles, "block_steps": r.iters,
                               "converged": bool(r.converged), "rel_res": r.rel_res.tolist(),
                               "rows": rows.tolist(), "x_ir": r.X[rows].tolist(),
                               "x_fp64": X64[rows].tolist(), "seconds": time.time() - t})
        print(s, A.n, r.cycles, r.converged, float(r.rel_res.max()), round(t_ir, 1), flush=True)
    with open(os.path.join(HERE, "oracle_batched_256.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
