"""The delayed classical Gram-Schmidt (DCGS2) variant against the CPU oracle (needs a GPU).

DCGS2 (params.orth = 1) is a different algorithm from the CGS2 of Section III-A: it merges each
step's second projection into the next step's first, one reduction per step.  The oracle's
gmres_cycle_dcgs2 follows the same steps; the tests compare the Hessenberg matrix and basis of
the FP64 kernels element by element, bound the FP32/BF16 ones, and compare whole solves (GMRES-IR
and FP64 GMRES, with and without the polynomial preconditioner) with the oracle's.
"""
import numpy as np
import pytest
import torch

import paper_2105_07544_b300 as g
import synth
from oracle import gmres as og
from gpu_util import dev, need_gpu, random_csr

pytestmark = pytest.mark.gpu


def _relres(A, b, x):
    return np.linalg.norm(b - og.spmv(A, x)) / np.linalg.norm(b)


def _dcgs2(s):
    s.set_params(orth=1)
    return s


@pytest.mark.parametrize("k", [1, 2, 9, 30])
def test_dcgs2_arnoldi_fp64_matches_oracle(k):
    need_gpu()
    A = synth.convdiff2d(60, 0.8, 100.0)          # n = 3600: 29 tiles, ragged tail
    r0 = synth.uniform(A.n, 5)
    s = _dcgs2(g.Solver(A, m=40))
    H, V, steps = s.arnoldi(dev(r0), k, "f64")
    assert steps == k
    co = og.gmres_cycle_dcgs2(lambda z: og.spmv(A, z), r0, k)
    Anorm = np.linalg.norm(A.val)
    assert np.max(np.abs(H - co.H)) <= 1e-11 * Anorm
    V = V.cpu().numpy()[:, :k]                     # column k is the candidate, not a basis vector
    assert np.max(np.abs(V - co.V[:, :k])) <= 1e-10
    if k > 1:
        AV = np.column_stack([og.spmv(A, V[:, i]) for i in range(k - 1)])
        assert np.linalg.norm(AV - V @ H[:k, :k - 1]) / Anorm <= 1e-13
    assert np.linalg.norm(np.eye(k) - V.T @ V) <= 1e-13
    s.close()


@pytest.mark.parametrize("name,mk", [
    ("laplace3d_17", lambda: synth.laplace3d(17)),
    ("random_longrows", lambda: random_csr(700, 4, 1, 6, dense_rows=(5, 300, 301), dense_len=690)),
])
def test_dcgs2_arnoldi_fp64_every_lane_shape(name, mk):
    """The reduction kernel's SpMV takes the lanes-per-row form for long rows."""
    need_gpu()
    A = mk()
    r0 = synth.uniform(A.n, 7)
    k = 12
    for lanes in (0, 4, 32):
        s = _dcgs2(g.Solver(A, m=20))
        s.set_tuning(spmv_lanes_per_row=lanes)
        H, V, steps = s.arnoldi(dev(r0), k, "f64")
        co = og.gmres_cycle_dcgs2(lambda z: og.spmv(A, z), r0, k)
        assert steps == co.k
        scale = np.abs(co.H).max()
        assert np.max(np.abs(H[: steps + 1, :steps] - co.H)) <= 1e-11 * scale
        s.close()


@pytest.mark.parametrize("basis,orth_tol,h_tol", [("f32", 1e-5, 2e-5), ("bf16", 5e-2, 2e-2)])
def test_dcgs2_arnoldi_low_precision_bounds(basis, orth_tol, h_tol):
    need_gpu()
    A = synth.laplace3d(17)
    r0 = synth.uniform(A.n, 6)
    k = 25
    s = _dcgs2(g.Solver(A, m=30, basis=basis))
    H, V, steps = s.arnoldi(dev(r0), k, "f32")
    assert steps == k
    co = og.gmres_cycle_dcgs2(lambda z: og.spmv(A, z), r0, k)
    Anorm = np.abs(A.val).max() * 7
    assert np.max(np.abs(H - co.H)) <= h_tol * Anorm
    V = V.cpu().numpy()[:, :k]
    assert np.linalg.norm(np.eye(k) - V.T @ V) <= orth_tol * k
    s.close()


def test_dcgs2_k_distinct_eigenvalues_and_exact_breakdown():
    """On k distinct eigenvalues the FP64 solve stops after exactly k iterations (implicit
    residual at tol; DCGS2's Pythagorean norm sqrt(alpha - s^T s) keeps only ~sqrt(u) of a
    near-breakdown, so the stop comes from the residual, as in the oracle).  An exact eigenvector
    leaves a zero candidate: an exact lucky breakdown after one step."""
    need_gpu()
    lam = np.array([0.5, 1.0, 2.0, 3.5, 5.0, 8.0, 13.0])
    d = np.repeat(lam, 40)
    A = synth.CSR(n=len(d), rowptr=np.arange(len(d) + 1, dtype=np.int32),
                  colidx=np.arange(len(d), dtype=np.int32), val=d)
    b = synth.uniform(A.n, 4)
    s = _dcgs2(g.Solver(A, m=20))
    x, st = s.solve_fp64(dev(b), tol=1e-12)
    assert st.converged and st.iters == len(lam)
    assert np.linalg.norm(x.cpu().numpy() - b / d) <= 1e-11 * np.linalg.norm(b / d)
    e = np.zeros(A.n)
    e[137] = 2.0
    H, V, steps = s.arnoldi(dev(e), 5, "f64")
    assert steps == 1 and H[0, 0] == d[137] and H[1, 0] == 0.0
    s.close()


@pytest.fixture(scope="module")
def c1():
    A, b, xstar = synth.workload_laplace2d_64()
    return A, b, og.gmres(A, b, 50, 1e-12), og.gmres_ir(A, b, 50, 1e-10, orth="dcgs2"), \
        og.gmres(A, b, 50, 1e-10, orth="dcgs2")


@pytest.mark.parametrize("basis", ["f32", "bf16"])
def test_dcgs2_gmres_ir_laplace2d_64(c1, basis):
    need_gpu()
    A, b, ref12, refir, _ = c1
    s = _dcgs2(g.Solver(A, m=50, basis=basis))
    x, st = s.ir_solve(dev(b), tol=1e-10)
    assert st.converged and _relres(A, b, x.cpu().numpy()) <= 1e-10
    assert st.iters % 50 == 0
    if basis == "f32":
        assert abs(st.cycles - refir.cycles) <= 1
    x12, st12 = s.ir_solve(dev(b), tol=1e-12)
    assert st12.converged
    assert np.linalg.norm(x12.cpu().numpy() - ref12.x) / np.linalg.norm(ref12.x) <= 1e-8
    s.close()


def test_dcgs2_fp64_gmres_laplace2d_64(c1):
    need_gpu()
    A, b, ref12, _, ref10 = c1
    s = _dcgs2(g.Solver(A, m=50))
    x, st = s.solve_fp64(dev(b), tol=1e-10)
    assert st.converged and _relres(A, b, x.cpu().numpy()) <= 1e-10
    assert abs(st.iters - ref10.iters) <= max(2, 0.01 * ref10.iters)
    s.close()


def test_dcgs2_ir_with_polynomial_against_oracle():
    need_gpu()
    A = synth.convdiff2d(120, 1.3, 100.0)
    b = synth.uniform(A.n, 9)
    start = synth.poly_start_vector(A.n, 0)
    P = og.poly_build(A, 10, start)
    ref = og.gmres_ir(A, b, 30, 1e-10, poly=P, orth="dcgs2")
    s = _dcgs2(g.Solver(A, m=30, poly_degree=10, poly_start=start))
    x, st = s.ir_solve(dev(b), tol=1e-10)
    assert st.converged and _relres(A, b, x.cpu().numpy()) <= 1e-10
    assert abs(st.cycles - ref.cycles) <= 1
    s.close()


def test_dcgs2_graphs_direct_launches_and_short_last_cycle(c1):
    """Graph replay and direct launches give the same iterate bit for bit; a maxiter that ends
    inside a cycle stops exactly there (the reduction kernel finishes the column at jmax)."""
    need_gpu()
    A, b, *_ = c1
    s = _dcgs2(g.Solver(A, m=50))
    x1, s1 = s.ir_solve(dev(b), tol=1e-10)
    s.set_params(use_graphs=0)
    x2, s2 = s.ir_solve(dev(b), tol=1e-10)
    s.set_params(profiling=1)
    x3, s3 = s.ir_solve(dev(b), tol=1e-10)
    assert torch.equal(x1, x2) and torch.equal(x1, x3)
    assert s3.t_kernel["spmv"] > 0 and s3.t_kernel["cgs_update"] > 0 and s3.t_kernel["cgs_proj"] > 0
    assert s3.t_kernel["cgs_pass2"] == 0
    s.set_params(use_graphs=1, profiling=0, maxiter=73)
    _, s4 = s.ir_solve(dev(b), tol=1e-10)
    assert s4.status == g.NOT_CONVERGED and s4.iters == 73
    s.close()


def test_dcgs2_refuses_the_scaled_fp16_basis(c1):
    need_gpu()
    A, b, *_ = c1
    s = _dcgs2(g.Solver(A, m=20, basis="f16"))
    with pytest.raises(g.GmresError):
        s.ir_solve(dev(b), tol=1e-10)
    s.close()
