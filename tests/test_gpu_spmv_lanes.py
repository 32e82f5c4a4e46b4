"""Lanes-per-row CSR SpMV (needs a GPU): on a matrix with long rows (60 nonzeros per row) every
lane count gives the oracle's products, and GMRES-IR and FP64 GMRES reach the oracle's solution
with each of them and with the automatic choice."""
import numpy as np
import pytest
import torch

import paper_2105_07544_b300 as g
import synth
from oracle import gmres as og
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu
M = 30
LANES = [1, 2, 4, 8, 16, 32]


@pytest.fixture(scope="module")
def long_rows():
    A = synth.random_rows(20000, 60, 3000, seed=1)
    b = synth.uniform(A.n, 3)
    ref = og.gmres_ir(A, b, M, 1e-10)
    assert ref.converged
    xs = og.gmres(A, b, M, 1e-13).x
    absA = synth.CSR(A.n, A.rowptr, A.colidx, np.abs(A.val))
    return A, b, ref, xs, absA


def _relres(A, b, x):
    return np.linalg.norm(b - og.spmv(A, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("lanes", LANES)
def test_spmv_each_lane_count_matches_the_oracle(long_rows, lanes):
    """Row sums of 60 products in another order: FP64 within 1e-13 and FP32 within 1e-5 of
    (|A| |x|)_i, row by row."""
    need_gpu()
    A, _, _, _, absA = long_rows
    s = g.Solver(A, m=M)
    s.set_tuning(spmv_lanes_per_row=lanes)
    xh = synth.uniform(A.n, 5)
    ref = og.spmv(A, xh)
    scale = og.spmv(absA, np.abs(xh))
    y64 = s.spmv(torch.from_numpy(xh).cuda(), "f64").cpu().numpy()
    assert np.all(np.abs(y64 - ref) <= 1e-13 * scale)
    x32 = xh.astype(np.float32)
    y32 = s.spmv(torch.from_numpy(x32).cuda(), "f32").cpu().numpy().astype(np.float64)
    ref32 = og.spmv(A, x32.astype(np.float64))
    assert np.all(np.abs(y32 - ref32) <= 1e-5 * scale)
    s.close()


@pytest.mark.parametrize("lanes", [0] + LANES)
def test_ir_solve_with_each_lane_count(long_rows, lanes):
    need_gpu()
    A, b, ref, xs, _ = long_rows
    s = g.Solver(A, m=M)
    s.set_tuning(spmv_lanes_per_row=lanes)
    assert s.get_tuning()["spmv_lanes_per_row"] == lanes
    x, st = s.ir_solve(torch.from_numpy(b).cuda(), tol=1e-10)
    s.close()
    x = x.cpu().numpy()
    assert st.converged and st.rel_res <= 1e-10 and _relres(A, b, x) <= 1e-10
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert abs(st.iters - ref.iters) <= M


@pytest.mark.parametrize("lanes", [1, 8])
def test_fp64_gmres_with_lanes(long_rows, lanes):
    need_gpu()
    A, b, _, xs, _ = long_rows
    ref = og.gmres(A, b, M, 1e-10)
    s = g.Solver(A, m=M)
    s.set_tuning(spmv_lanes_per_row=lanes)
    x, st = s.solve_fp64(torch.from_numpy(b).cuda(), tol=1e-10)
    s.close()
    assert st.converged and _relres(A, b, x.cpu().numpy()) <= 1e-10
    assert abs(st.iters - ref.iters) <= 1


def test_invalid_lane_counts_are_rejected():
    need_gpu()
    s = g.Solver(synth.laplace2d(16), m=10)
    for bad in (3, 64, -1):
        with pytest.raises(g.GmresError):
            s.set_tuning(spmv_lanes_per_row=bad)
    s.close()
