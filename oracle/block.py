"""CPU oracle for block GMRES(m) and block GMRES-IR with p right-hand sides (batched workload).

TEST INFRASTRUCTURE ONLY (see oracle/gmres.py for the rules).  The block method applies
Algorithm 1 to a block of p vectors: the Krylov space of A and the block R0 is built with block
classical Gram-Schmidt run twice (block CGS2, Section III-A's CGS2 with V_j^T W a dense product),
each new block orthonormalised by a Cholesky QR, and the least-squares problem
min ||E1 B0 - Hbar Y||_F solved once per cycle.  Block GMRES-IR follows Algorithm 2 per block:
FP64 residual and update, one FP32 cycle per refinement step.

Readings (where the paper, which has no block method, is silent):
* The p columns of the residual are scaled to unit norm before the first QR (R0 = R D^{-1}),
  so converged and unconverged columns do not make the Gram matrix singular.
* Cholesky QR: G = W^T W = L L^T, Q = W L^{-T}, the new Hessenberg block is L^T.  If G is not
  numerically positive definite, a shift 11 (n p + p(p+1)) u ||G|| is added once (shifted
  Cholesky QR); if that fails too, the cycle ends.
* With a BF16 basis the stored block is bf16(W) and the QR is taken of the stored block, so the
  orthonormal block is bf16(W) L^{-T}.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .gmres import F32, F64, round_bf16, spmv, unit_roundoff


def spmm(A, X, dtype=F64):
    """Y = A X for a block of columns (column by column with the oracle's SpMV)."""
    X = np.asarray(X, dtype=dtype)
    return np.column_stack([spmv(A, X[:, c], dtype) for c in range(X.shape[1])])


def chol_qr(W, dtype, basis_round=None):
    """Stored block U, orthonormal Q = U L^{-T} and R = L^T with U^T U = L L^T (shifted if needed)."""
    U = basis_round(W) if basis_round else np.asarray(W, dtype=dtype)
    G = (U.T @ U).astype(F64)
    n, p = U.shape
    try:
        L = np.linalg.cholesky(G)
    except np.linalg.LinAlgError:
        shift = 11.0 * (n * p + p * (p + 1)) * unit_roundoff(dtype) * np.linalg.norm(G, 2)
        L = np.linalg.cholesky(G + shift * np.eye(p))
    Q = (U.astype(F64) @ np.linalg.inv(L).T).astype(dtype)
    return U, Q, L.T.astype(dtype)


@dataclass
class BlockCycle:
    X: np.ndarray        # correction V Y (n x p)
    H: np.ndarray        # block Hessenberg ((k+1)p x kp)
    V: np.ndarray        # orthonormal basis (n x (k+1)p)
    k: int
    implicit: list = field(default_factory=list)   # per step: column residual norms of the LS


def block_gmres_cycle(apply_op, R0, m, dtype=F64, basis_round=None):
    """m steps of block Arnoldi with block CGS2 from the block R0 (n x p)."""
    n, p = R0.shape
    _, Q, B0 = chol_qr(R0, dtype, basis_round)
    Qs = [Q]
    H = np.zeros(((m + 1) * p, m * p), dtype=F64)
    imp = []
    k = 0
    for j in range(m):
        W = np.asarray(apply_op(Qs[j]), dtype=dtype)
        Vj = np.hstack(Qs)
        for _ in range(2):                                   # block CGS2
            Hj = Vj.T @ W
            W = W - Vj @ Hj
            H[: (j + 1) * p, j * p:(j + 1) * p] += Hj
        try:
            _, Qn, Rn = chol_qr(W, dtype, basis_round)
        except np.linalg.LinAlgError:
            break
        H[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = Rn
        Qs.append(Qn)
        k = j + 1
        Hk = H[: (k + 1) * p, : k * p]
        E = np.zeros(((k + 1) * p, p))
        E[:p] = B0
        Y, *_ = np.linalg.lstsq(Hk, E, rcond=None)
        imp.append(np.linalg.norm(E - Hk @ Y, axis=0))
    Hk = H[: (k + 1) * p, : k * p]
    E = np.zeros(((k + 1) * p, p))
    E[:p] = B0
    Y, *_ = np.linalg.lstsq(Hk, E, rcond=None)
    V = np.hstack(Qs)
    X = V[:, : k * p].astype(F64) @ Y
    return BlockCycle(X=X, H=Hk, V=V, k=k, implicit=imp)


@dataclass
class BlockResult:
    X: np.ndarray
    iters: int
    cycles: int
    rel_res: np.ndarray      # per column ||b - A x|| / ||b||
    converged: bool
    history: list = field(default_factory=list)


def block_gmres_ir(A, B, m, tol, basis="f32", maxcycles=500, dtype_inner=F32):
    """Block GMRES-IR: FP64 residual and update, one block cycle in FP32 per refinement step."""
    B = np.asarray(B, dtype=F64)
    X = np.zeros_like(B)
    bn = np.linalg.norm(B, axis=0)
    rnd = round_bf16 if basis == "bf16" else None
    op = lambda Z: spmm(A, Z, dtype_inner)
    res = BlockResult(X=X, iters=0, cycles=0, rel_res=None, converged=False)
    for _ in range(maxcycles + 1):
        R = B - spmm(A, X)
        rel = np.linalg.norm(R, axis=0) / bn
        res.history.append(rel.copy())
        res.rel_res = rel
        if np.all(rel <= tol):
            res.converged = True
            break
        if res.cycles >= maxcycles:
            break
        D = np.linalg.norm(R, axis=0)
        cyc = block_gmres_cycle(op, (R / D).astype(dtype_inner), m, dtype_inner, rnd)
        X = X + cyc.X * D                     # the inner system was scaled column-wise by 1/D
        res.iters += cyc.k
        res.cycles += 1
    res.X = X
    return res
