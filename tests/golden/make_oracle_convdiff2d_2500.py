"""Write oracle_convdiff2d_2500_<mode>.json: the CPU oracle's solves of the 2D upwind
convection-diffusion problem 2500^2 (n = 6,250,000; theta ~ U[0, 2 pi) and b ~ U[-1,1) from seed
0, Peclet 100) right-preconditioned by the degree-25 GMRES polynomial (built in FP64 from the
seeded start vector), GMRES(50), tol 1e-10.  Calls only oracle/ and synth/.

    python tests/golden/make_oracle_convdiff2d_2500.py ir-bf16|ir-f32|fp64

ir-bf16 / ir-f32: GMRES-IR (Algorithm 2) with the polynomial applied in FP32 and the Krylov basis
stored in BF16 / FP32.  fp64: FP64 GMRES (Algorithm 1) with the polynomial in FP64.  Stored:
iteration and cycle counts, the final explicit residual, the per-cycle explicit residual history,
x at 64 seeded sample rows and the Leja-ordered polynomial roots.  Each mode takes about an hour
on one host core.
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

N, DEGREE, M, TOL = 2500, 25, 50, 1e-10


def main(mode):
    A, b, theta = synth.workload_convdiff2d(N, 0)
    pstart = synth.poly_start_vector(A.n, 0)
    rows = np.sort(np.random.default_rng(123).choice(A.n, 64, replace=False))
    t = time.time()
    P = og.poly_build(A, DEGREE, pstart)
    out = {"_source": "tests/golden/make_oracle_convdiff2d_2500.py (oracle only)",
           "workload": f"convdiff2d_{N}, theta = {theta!r}, Pe 100, b ~ U[-1,1) seed 0, "
                       f"degree-{DEGREE} GMRES polynomial, m = {M}, tol {TOL}, mode {mode}",
           "sample_rows": rows.tolist(),
           "roots_re": P.roots.real.tolist(), "roots_im": P.roots.imag.tolist(),
           "poly_build_seconds": time.time() - t}
    t = time.time()
    if mode == "fp64":
        r = og.gmres(A, b, M, TOL, poly=P)
    else:
        r = og.gmres_ir(A, b, M, TOL, poly=P, basis=mode.split("-")[1])
    out["result"] = {"iters": r.iters, "cycles": r.cycles, "rel_res": r.rel_res,
                     "converged": bool(r.converged), "history": r.history,
                     "x_sample": r.x[rows].tolist(), "seconds": time.time() - t}
    print(mode, r.iters, r.cycles, r.rel_res, time.time() - t, flush=True)
    with open(os.path.join(HERE, f"oracle_convdiff2d_{N}_{mode}.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    if len(sys.argv) != 2 or sys.argv[1] not in ("ir-bf16", "ir-f32", "fp64"):
        sys.exit(__doc__)
    main(sys.argv[1])
