"""Pins of the block-GMRES oracle (no GPU): reduction to the scalar oracle at p = 1, the block
Arnoldi relation, exact termination, full-space solves against LAPACK, and convergence of block
GMRES-IR."""
import numpy as np
import pytest

import synth
from oracle import block as ob
from oracle import gmres as og


def _diag_csr(d):
    n = len(d)
    return synth.CSR(n=n, rowptr=np.arange(n + 1, dtype=np.int32),
                     colidx=np.arange(n, dtype=np.int32), val=np.asarray(d, float))


def test_block_size_one_equals_scalar_oracle():
    A = synth.convdiff2d(30, 0.6, 100.0, 0.1)
    b = synth.uniform(A.n, 3)
    cyc = ob.block_gmres_cycle(lambda Z: ob.spmm(A, Z), b[:, None], 20)
    sc = og.gmres_cycle(lambda z: og.spmv(A, z), b, 20)
    assert cyc.k == sc.k == 20
    assert np.allclose(cyc.H, sc.H, rtol=0, atol=1e-12)
    xs = sc.V[:, : sc.k] @ sc.y
    assert np.linalg.norm(cyc.X[:, 0] - xs) <= 1e-12 * np.linalg.norm(xs)


def test_block_arnoldi_relation_and_orthogonality():
    A = synth.convdiff2d(24, 2.0, 100.0, 0.3)
    R0 = np.random.default_rng(1).uniform(-1, 1, (A.n, 8))
    cyc = ob.block_gmres_cycle(lambda Z: ob.spmm(A, Z), R0, 6)
    p, k = 8, cyc.k
    V = cyc.V
    assert V.shape == (A.n, (k + 1) * p)
    assert np.linalg.norm(np.eye((k + 1) * p) - V.T @ V) <= 1e-12
    AV = ob.spmm(A, V[:, : k * p])
    assert np.linalg.norm(AV - V @ cyc.H) <= 1e-12 * np.linalg.norm(A.val)
    # block upper Hessenberg: blocks below the first block subdiagonal vanish, subdiagonal
    # blocks are upper triangular (Cholesky QR)
    for j in range(k):
        assert np.all(cyc.H[(j + 2) * p:, j * p:(j + 1) * p] == 0)
        sub = cyc.H[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p]
        assert np.allclose(np.tril(sub, -1), 0) and np.all(np.diag(sub) > 0)


def test_block_exact_termination():
    """With p right-hand sides the block Krylov space grows by p per step: on a matrix with d
    simple eigenvalues it is the whole space after ceil(d/p) steps and the solve is exact."""
    lam = np.array([0.5, 1.0, 2.0, 3.5, 5.0, 8.0, 13.0, 21.0, 34.0, 55.0, 89.0, 144.0])
    A = _diag_csr(lam)
    B = np.random.default_rng(2).uniform(-1, 1, (A.n, 4))
    cyc = ob.block_gmres_cycle(lambda Z: ob.spmm(A, Z), B, 3)   # 3 steps x 4 = 12 = n
    assert np.linalg.norm(cyc.X - B / lam[:, None]) <= 1e-9 * np.linalg.norm(B)
    two = ob.block_gmres_cycle(lambda Z: ob.spmm(A, Z), B, 2)   # 8 < 12: not yet exact
    assert np.linalg.norm(two.X - B / lam[:, None]) > 1e-6 * np.linalg.norm(B)


def test_block_full_space_equals_direct_solve():
    rng = np.random.default_rng(4)
    n = 48
    M = rng.standard_normal((n, n)) + 0.4 * n * np.eye(n)
    rows, cols = np.nonzero(M)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    A = synth.CSR(n=n, rowptr=np.cumsum(rowptr).astype(np.int32), colidx=cols.astype(np.int32),
                  val=M[rows, cols])
    B = rng.standard_normal((n, 4))
    cyc = ob.block_gmres_cycle(lambda Z: ob.spmm(A, Z), B, n // 4)
    Xd = np.linalg.solve(M, B)
    assert np.linalg.norm(cyc.X - Xd) <= np.linalg.cond(M) * 1e-13 * np.linalg.norm(Xd)


def test_chol_qr_factorisation():
    W = np.random.default_rng(5).standard_normal((300, 8))
    U, Q, R = ob.chol_qr(W, np.float64)
    assert np.allclose(Q.T @ Q, np.eye(8), atol=1e-12)
    assert np.allclose(Q @ R, W, atol=1e-12)
    Ub, Qb, Rb = ob.chol_qr(W.astype(np.float32), np.float32, og.round_bf16)
    assert np.array_equal(Ub, og.round_bf16(W.astype(np.float32)))
    assert np.linalg.norm(Qb.T @ Qb - np.eye(8)) <= 1e-4


@pytest.mark.parametrize("dtype,rtol", [(np.float64, 1e-12), (np.float32, 1e-6)])
def test_chol_qr_shifted_branch_on_a_rank_deficient_block(dtype, rtol):
    """A block with a zero column has an exactly singular Gram matrix (a zero pivot), so the plain
    Cholesky factorisation fails and the shifted one runs: U^T U + s I = R^T R with
    s = 11 (n p + p (p + 1)) u ||G||_2 (shifted Cholesky QR, Fukaya et al. 2020).  The zero
    column's pivot is sqrt(s) exactly; the other columns come out orthonormal."""
    rng = np.random.default_rng(7)
    n, p, k = 200, 8, 5
    W = rng.standard_normal((n, p)).astype(dtype)
    W[:, k] = 0.0
    with pytest.raises(np.linalg.LinAlgError):
        np.linalg.cholesky((W.T @ W).astype(np.float64))
    U, Q, R = ob.chol_qr(W, dtype)
    G = (U.T @ U).astype(np.float64)
    u = np.finfo(dtype).eps / 2
    s = 11.0 * (n * p + p * (p + 1)) * u * np.linalg.norm(G, 2)
    R64 = R.astype(np.float64)
    assert abs(R64[k, k] ** 2 - s) <= rtol * s
    assert np.allclose(R64.T @ R64, G + s * np.eye(p), rtol=0, atol=rtol * np.linalg.norm(G, 2))
    assert not np.any(Q[:, k])
    keep = [c for c in range(p) if c != k]
    Qk = Q[:, keep].astype(np.float64)
    assert np.linalg.norm(Qk.T @ Qk - np.eye(p - 1)) <= 1e3 * s / np.linalg.norm(G, 2) + 10 * rtol
    # two equal columns: the shifted branch or a tiny pivot, never a failure; Q R = W still holds
    W2 = rng.standard_normal((n, p)).astype(dtype)
    W2[:, 3] = W2[:, 2]
    U2, Q2, R2 = ob.chol_qr(W2, dtype)
    assert np.all(np.isfinite(Q2)) and np.all(np.isfinite(R2))
    err = np.linalg.norm(Q2.astype(np.float64) @ R2.astype(np.float64) - W2)
    assert err <= 1e3 * np.sqrt(s) * np.sqrt(p) + 1e-3 * rtol * np.linalg.norm(W2)


@pytest.mark.parametrize("basis", ["f32", "bf16"])
def test_block_gmres_ir_converges_per_column(basis):
    A = synth.convdiff2d(40, 1.0, 100.0, shift=0.2)
    B = np.random.default_rng(0).uniform(-1, 1, (A.n, 8))
    r = ob.block_gmres_ir(A, B, 10, 1e-10, basis=basis)
    assert r.converged and np.all(r.rel_res <= 1e-10)
    X = np.column_stack([og.gmres(A, B[:, c], 60, 1e-12).x for c in range(8)])
    assert np.linalg.norm(r.X - X) <= 1e-7 * np.linalg.norm(X)


def test_block_residuals_are_monotone_and_match_the_explicit_ones():
    """Within a cycle each column's least-squares residual cannot grow (the block Krylov space
    only grows), and in FP64 it equals the explicit residual ||R0 - A X|| of that column."""
    A = synth.convdiff2d(26, 1.1, 100.0, 0.2)
    R0 = np.random.default_rng(5).uniform(-1.0, 1.0, (A.n, 8))
    cyc = ob.block_gmres_cycle(lambda Z: ob.spmm(A, Z), R0, 12)
    imp = np.array(cyc.implicit)                   # [step][column]
    assert imp.shape == (12, 8)
    assert np.all(imp[1:] <= imp[:-1] * (1 + 1e-12))
    assert np.all(imp[-1] < 0.5 * np.linalg.norm(R0, axis=0))
    explicit = np.linalg.norm(R0 - ob.spmm(A, cyc.X), axis=0)
    assert np.allclose(explicit, imp[-1], rtol=1e-9, atol=0)
