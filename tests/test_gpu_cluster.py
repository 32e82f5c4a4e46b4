"""The cluster-resident restart cycle of small systems (needs a GPU).

A system whose basis fits in the shared memory of at most 16 CTAs runs each restart cycle as one
kernel on one thread-block cluster (`gmres_tuning_t.cluster_cycle = 0`, the default).  These
tests check it against the CPU oracle (Algorithms 1 and 2 with CGS2) and against the per-step
kernels (`cluster_cycle = -1`), and that it is the path that ran: a solve on it launches one
kernel per cycle plus the two of its set-up (||b|| and the first residual)."""
import numpy as np
import pytest
import torch

import paper_2105_07544_b300 as g
import synth
from oracle import gmres as og
from gpu_util import dev, need_gpu

pytestmark = pytest.mark.gpu


def _relres(A, b, x):
    return np.linalg.norm(b - og.spmv(A, x)) / np.linalg.norm(b)


def _solve(A, b, solve, cluster, m=50, tol=1e-10, **params):
    s = g.Solver(A, m=m)
    if not cluster:
        s.set_tuning(cluster_cycle=-1)
    if params:
        s.set_params(**params)
    x, st = getattr(s, solve)(dev(b), tol=tol)
    s.close()
    return x.cpu().numpy(), st


def _random_sparse(n, seed, band=3):
    """Nonsymmetric, diagonally dominant, `band` off-diagonals on each side (unsorted rows)."""
    rng = np.random.default_rng(seed)
    M = np.diag(4.0 + rng.uniform(0, 1, n))
    for k in range(1, band + 1):
        M += np.diag(rng.uniform(-1, 1, n - k), k) + np.diag(rng.uniform(-1, 1, n - k), -k)
    rows, cols = np.nonzero(M)
    order = rng.permutation(len(rows))                  # columns unsorted within a row
    order = order[np.argsort(rows[order], kind="stable")]
    rows, cols = rows[order], cols[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return synth.CSR(n=n, rowptr=np.cumsum(rp).astype(np.int32), colidx=cols.astype(np.int32),
                     val=M[rows, cols])


@pytest.fixture(scope="module")
def c1():
    A, b, _ = synth.workload_laplace2d_64()
    return (A, b, og.gmres(A, b, m=50, tol=1e-10), og.gmres(A, b, m=50, tol=1e-12),
            og.gmres_ir(A, b, m=50, tol=1e-10))


def test_fp64_gmres_on_one_cluster_matches_the_oracle(c1):
    """64^2 Laplacian (n = 4096: 16 CTAs of 256 rows): the oracle's iteration count, the
    solution to 1e-8 at tol 1e-10 (against the oracle's own 1e-10 iterate) and at tol 1e-12
    (against its 1e-12 solution), one launch per cycle."""
    need_gpu()
    A, b, ref10, ref12, _ = c1
    x, st = _solve(A, b, "solve_fp64", True)
    assert st.converged and st.rel_res <= 1e-10 and _relres(A, b, x) <= 1e-10
    assert st.kernel_launches == st.cycles + 2
    assert abs(st.iters - ref10.iters) <= max(2, 0.01 * ref10.iters)
    assert np.linalg.norm(x - ref10.x) / np.linalg.norm(ref10.x) <= 1e-8
    assert st.loss_of_accuracy == 0
    x12, st12 = _solve(A, b, "solve_fp64", True, tol=1e-12)
    assert st12.converged and np.linalg.norm(x12 - ref12.x) / np.linalg.norm(ref12.x) <= 1e-8


def test_gmres_ir_on_one_cluster_matches_the_oracle(c1):
    """FP32 inner cycles, FP64 residual and update: the oracle's cycle count, the FP64 residual
    recomputed by the oracle, the 1e-12 solution against the oracle's."""
    need_gpu()
    A, b, _, ref12, refir = c1
    x, st = _solve(A, b, "ir_solve", True)
    assert st.converged and _relres(A, b, x) <= 1e-10
    assert st.kernel_launches == st.cycles + 2
    assert st.iters % 50 == 0 and abs(st.cycles - refir.cycles) <= 1
    x12, st12 = _solve(A, b, "ir_solve", True, tol=1e-12)
    assert st12.converged and _relres(A, b, x12) <= 1e-12
    assert np.linalg.norm(x12 - ref12.x) / np.linalg.norm(ref12.x) <= 1e-8


def test_gmres_ir_bf16_basis_on_one_cluster_matches_the_oracle(c1):
    """BF16 basis (FP32 arithmetic, FP64 residual): the oracle's BF16 GMRES-IR cycle count, the
    FP64 residual recomputed by the oracle, and the 1e-12 solution against the oracle's."""
    need_gpu()
    A, b, _, ref12, _ = c1
    refb = og.gmres_ir(A, b, m=50, tol=1e-10, basis="bf16")
    s = g.Solver(A, m=50, basis="bf16")
    x, st = s.ir_solve(dev(b), tol=1e-10)
    assert st.converged and _relres(A, b, x.cpu().numpy()) <= 1e-10
    assert st.kernel_launches == st.cycles + 2
    assert abs(st.cycles - refb.cycles) <= 1
    x12, st12 = s.ir_solve(dev(b), tol=1e-12)
    assert st12.converged and _relres(A, b, x12.cpu().numpy()) <= 1e-12
    assert np.linalg.norm(x12.cpu().numpy() - ref12.x) / np.linalg.norm(ref12.x) <= 1e-8
    s.close()


@pytest.mark.parametrize("solve", ["solve_fp64", "ir_solve"])
def test_cluster_and_step_kernels_agree(c1, solve):
    """Same algorithm, different summation order: the two paths end within an iteration (FP64)
    or a cycle (IR) of each other, on solutions that agree within what a 1e-10 residual fixes
    (kappa * 1e-10, kappa ~ 1.7e3 here)."""
    need_gpu()
    A, b, *_ = c1
    xc, sc = _solve(A, b, solve, True)
    xs, ss = _solve(A, b, solve, False)
    assert sc.converged and ss.converged
    assert ss.kernel_launches > 10 * ss.cycles
    if solve == "solve_fp64":
        assert abs(sc.iters - ss.iters) <= 1
    else:
        assert abs(sc.cycles - ss.cycles) <= 1
    assert np.linalg.norm(xc - xs) / np.linalg.norm(xs) <= 1e-6
    assert sc.rel_res_implicit > 0


@pytest.mark.parametrize("name,mk,solves", [
    # 45^2 = 2025 rows: 8 CTAs, the last one ragged (233 rows)
    ("laplace2d_45", lambda: synth.laplace2d(45), ("solve_fp64", "ir_solve")),
    # 4900 rows: 10 CTAs of 512 rows (FP32 and, at m = 30, FP64 basis)
    ("convdiff_70", lambda: synth.convdiff2d(70, 2.2, 100.0), ("solve_fp64", "ir_solve")),
    # one CTA, unsorted columns, seven nonzeros per row
    ("random_200", lambda: _random_sparse(200, 11), ("solve_fp64", "ir_solve")),
])
def test_cluster_shapes_against_the_oracle(name, mk, solves):
    need_gpu()
    A = mk()
    b = synth.uniform(A.n, 21)
    for solve in solves:
        x, st = _solve(A, b, solve, True, m=30)
        assert st.converged and _relres(A, b, x) <= 1e-10, (solve, st.status)
        assert st.kernel_launches == st.cycles + 2, (solve, st.kernel_launches, st.cycles)
        if solve == "solve_fp64":
            ref = og.gmres(A, b, m=30, tol=1e-10)
            assert abs(st.iters - ref.iters) <= max(1, 0.01 * ref.iters)
            assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-7
        else:
            ref = og.gmres_ir(A, b, m=30, tol=1e-10)
            assert abs(st.cycles - ref.cycles) <= 1


def test_systems_that_do_not_fit_take_the_step_kernels():
    """The FP64 basis of 4900 rows at m = 50 needs more than 16 CTAs of 256 rows, or more shared
    memory than a CTA has at 512 rows (51 x 512 x 8 bytes): the per-step kernels run (many
    launches per cycle), with the oracle's iteration count."""
    need_gpu()
    A = synth.convdiff2d(70, 2.2, 100.0)
    b = synth.uniform(A.n, 21)
    x, st = _solve(A, b, "solve_fp64", True, m=50)
    assert st.converged and _relres(A, b, x) <= 1e-10
    assert st.kernel_launches > 10 * st.cycles
    ref = og.gmres(A, b, m=50, tol=1e-10)
    assert abs(st.iters - ref.iters) <= max(2, 0.01 * ref.iters)


def test_breakdown_stop_rules_and_resume_on_one_cluster():
    """An eigenvector right-hand side ends the first cycle by a lucky breakdown after one step;
    a short last cycle (maxiter not a multiple of m) stops the cluster's step loop early; the
    iterate of a capped solve resumes to the uncapped solve's count."""
    need_gpu()
    N = 20
    A = synth.laplace2d(N)
    i = np.arange(1, N + 1)
    v = np.outer(np.sin(3 * np.pi * i / (N + 1)), np.sin(2 * np.pi * i / (N + 1))).ravel()
    x, st = _solve(A, v, "solve_fp64", True, m=10)
    assert st.converged and st.iters == 1 and _relres(A, v, x) <= 1e-10
    A, b, _ = synth.workload_laplace2d_64()
    s = g.Solver(A, m=50)
    s.set_params(maxiter=73)
    xp, stp = s.solve_fp64(dev(b), tol=1e-10)
    assert stp.status == g.NOT_CONVERGED and stp.iters == 73 and stp.cycles == 2
    s.set_params(maxiter=200000)
    xr, str_ = s.solve_fp64(dev(b), x=xp.clone(), tol=1e-10)
    assert str_.converged and _relres(A, b, xr.cpu().numpy()) <= 1e-10
    assert str_.kernel_launches == str_.cycles + 2
    s.close()


def test_zero_and_converged_right_hand_sides_on_one_cluster():
    need_gpu()
    A, b, _ = synth.workload_laplace2d_64()
    x, st = _solve(A, np.zeros(A.n), "ir_solve", True)
    assert st.converged and not np.any(x)
    s = g.Solver(A, m=50)
    x1, st1 = s.solve_fp64(dev(b), tol=1e-10)
    x2, st2 = s.solve_fp64(dev(b), x=x1.clone(), tol=1e-10)   # already converged: no cycle
    assert st2.converged and st2.iters == 0 and torch.equal(x1, x2)
    s.close()


def test_cluster_cycle_setting_is_validated_and_kept_by_the_autotuner():
    """Only 0 (cluster when the system qualifies) and -1 (per-step kernels) are accepted; the
    autotuner times the per-step kernels' launch shapes and leaves the setting as it was."""
    need_gpu()
    A, b, _ = synth.workload_laplace2d_64()
    s = g.Solver(A, m=50)
    for bad in (1, -2):
        with pytest.raises(g.GmresError):
            s.set_tuning(cluster_cycle=bad)
    s.set_tuning(cluster_cycle=-1)
    s.autotune(dev(b), cycles=1)
    x, st = s.ir_solve(dev(b), tol=1e-10)
    assert st.converged and st.kernel_launches > 10 * st.cycles     # still the per-step kernels
    s.set_tuning(cluster_cycle=0)
    s.autotune(dev(b), cycles=1)
    x, st = s.ir_solve(dev(b), tol=1e-10)
    assert st.converged and st.kernel_launches == st.cycles + 2     # back on the cluster
    s.close()
