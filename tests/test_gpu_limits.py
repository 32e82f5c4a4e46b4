"""The largest and the smallest shapes the library accepts, against the oracle (needs a GPU).

The restart length m = 127 fills every basis and partial-sum slot (128 columns): the Arnoldi
factorisation of 127 FP64 steps (CGS2 and DCGS2) matches the oracle's over its first 30 columns
and satisfies the Arnoldi relation and orthogonality throughout, and GMRES-IR with m = 127 runs in
every basis precision.  GMRES(1), a system smaller than
one 128-row tile and the degenerate right-hand sides are covered for both orthogonalisations.
"""
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


@pytest.mark.parametrize("orth", [0, 1])
def test_arnoldi_127_steps_fp64(orth):
    """127 FP64 Arnoldi steps: the first 30 columns of H equal the oracle's element by element
    (later ones amplify the two sides' different summation orders once the Krylov space nears an
    invariant subspace: both are backward stable, not forward-identical), and the whole
    factorisation satisfies the Arnoldi relation and orthogonality at FP64 level."""
    need_gpu()
    A = synth.convdiff2d(45, 0.6, 100.0)                  # n = 2025: 16 tiles, ragged tail
    r0 = synth.uniform(A.n, 12)
    k = 127
    s = g.Solver(A, m=127)
    s.set_params(orth=orth)
    H, V, steps = s.arnoldi(dev(r0), k, "f64")
    assert steps == k
    op = lambda z: og.spmv(A, z)
    co = og.gmres_cycle(op, r0, 30) if orth == 0 else og.gmres_cycle_dcgs2(op, r0, 30)
    Anorm = np.linalg.norm(A.val)
    assert np.max(np.abs(H[:31, :30] - co.H)) <= 1e-11 * Anorm
    V = V.cpu().numpy()[:, :k]                              # column k: the DCGS2 candidate
    AV = np.column_stack([og.spmv(A, V[:, i]) for i in range(k - 1)])
    assert np.linalg.norm(AV - V @ H[:k, :k - 1]) <= 1e-13 * np.sqrt(k) * Anorm
    assert np.linalg.norm(np.eye(k) - V.T @ V) <= 1e-12
    s.close()


@pytest.mark.parametrize("basis,orth", [("f32", 0), ("bf16", 0), ("f16", 0), ("f32", 1), ("bf16", 1)])
def test_gmres_ir_with_the_largest_restart(basis, orth):
    need_gpu()
    A = synth.convdiff2d(90, 1.9, 100.0)
    b = synth.uniform(A.n, 13)
    s = g.Solver(A, m=127, basis=basis)
    s.set_params(orth=orth)
    x, st = s.ir_solve(dev(b), tol=1e-10)
    assert st.converged and _relres(A, b, x.cpu().numpy()) <= 1e-10
    assert st.iters % 127 == 0
    if basis == "f32":
        ref = og.gmres_ir(A, b, 127, 1e-10, orth="dcgs2" if orth else "cgs2")
        assert abs(st.cycles - ref.cycles) <= 1
    s.close()


@pytest.mark.parametrize("orth", [0, 1])
def test_gmres_1_and_a_system_smaller_than_one_tile(orth):
    """GMRES(1) (one Arnoldi step per cycle) on a diagonally dominant system, and a 37-row
    system (one partial tile) solved exactly by a full Krylov space, against the oracle."""
    need_gpu()
    rng = np.random.default_rng(3)
    n = 300
    M = np.diag(4.0 + rng.uniform(0, 1, n)) + np.diag(rng.uniform(-1, 1, n - 1), 1) + \
        np.diag(rng.uniform(-1, 1, n - 1), -1)
    rows, cols = np.nonzero(M)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    A = synth.CSR(n=n, rowptr=np.cumsum(rp).astype(np.int32), colidx=cols.astype(np.int32),
                  val=M[rows, cols])
    b = synth.uniform(n, 4)
    ref = og.gmres(A, b, 1, 1e-10, orth="dcgs2" if orth else "cgs2")
    s = g.Solver(A, m=1)
    s.set_params(orth=orth)
    x, st = s.solve_fp64(dev(b), tol=1e-10)
    assert st.converged and _relres(A, b, x.cpu().numpy()) <= 1e-10
    assert abs(st.iters - ref.iters) <= max(2, 0.01 * ref.iters)
    xi, sti = s.ir_solve(dev(b), tol=1e-10)
    assert sti.converged and _relres(A, b, xi.cpu().numpy()) <= 1e-10
    s.close()
    # 37 rows, m = 50 > n: the Krylov space is the whole space after at most 37 steps
    n2 = 37
    M2 = rng.standard_normal((n2, n2)) + 0.5 * n2 * np.eye(n2)
    rows, cols = np.nonzero(M2)
    rp = np.zeros(n2 + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    A2 = synth.CSR(n=n2, rowptr=np.cumsum(rp).astype(np.int32), colidx=cols.astype(np.int32),
                   val=M2[rows, cols])
    b2 = synth.uniform(n2, 5)
    s = g.Solver(A2, m=50)
    s.set_params(orth=orth)
    x2, st2 = s.solve_fp64(dev(b2), tol=1e-13)
    assert st2.converged and st2.iters <= n2
    xs = np.linalg.solve(M2, b2)
    assert np.linalg.norm(x2.cpu().numpy() - xs) <= np.linalg.cond(M2) * 1e-13 * np.linalg.norm(xs)
    s.close()


def test_degenerate_right_hand_sides_with_dcgs2():
    """b = 0 gives x = 0; a NaN in b is reported; a converged initial guess takes no cycle."""
    need_gpu()
    A = synth.laplace2d(9)
    b = synth.uniform(A.n, 1)
    s = g.Solver(A, m=20)
    s.set_params(orth=1)
    x, st = s.ir_solve(dev(np.zeros(A.n)), tol=1e-10)
    assert st.converged and torch.count_nonzero(x).item() == 0
    bn = b.copy()
    bn[5] = np.nan
    _, st = s.ir_solve(dev(bn), tol=1e-10)
    assert st.status == g.NAN
    x, st = s.ir_solve(dev(b), tol=1e-12)
    x2, st2 = s.ir_solve(dev(b), x=x.clone(), tol=1e-10)
    assert st2.converged and st2.cycles == 0 and torch.equal(x2, x)
    s.close()
