"""Kernel-level parity of the CUDA path against the CPU oracle (needs a GPU).

SpMV, Arnoldi/CGS2 (Hessenberg entries, Arnoldi relation, orthogonality) and the polynomial
preconditioner are compared element by element with the oracle on the same seeded inputs, at
sizes that span several 128-row tiles and a ragged last tile.
"""
import numpy as np
import pytest
import torch

import paper_2105_07544_b300 as g
import synth
from oracle import gmres as og
from gpu_util import dev, need_gpu, random_csr

pytestmark = pytest.mark.gpu

U32 = 2.0**-24


def _absrow(A, x):
    """|A| |x| row sums (the scale of the SpMV rounding bound)."""
    import scipy.sparse as sp
    M = sp.csr_matrix((np.abs(A.val), A.colidx, A.rowptr), shape=(A.n, A.n))
    return M @ np.abs(x)


CASES = [
    ("laplace2d_64", lambda: synth.laplace2d(64)),
    ("laplace3d_19", lambda: synth.laplace3d(19)),            # n = 6859, ragged last tile
    ("convdiff_201", lambda: synth.convdiff2d(201, 2.0, 100.0)),
    ("random_ragged", lambda: random_csr(1000, 3, 0, 12)),    # empty rows, varied lengths
    ("random_longrows", lambda: random_csr(700, 4, 1, 6, dense_rows=(5, 300, 301), dense_len=690)),
    ("tiny_n1", lambda: synth.CSR(n=1, rowptr=np.array([0, 1], np.int32),
                                  colidx=np.array([0], np.int32), val=np.array([2.5]))),
]


@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_spmv_f64_and_f32(name, mk):
    need_gpu()
    A = mk()
    s = g.Solver(A, m=4)
    x = synth.uniform(A.n, 11)
    y64 = s.spmv(dev(x), "f64").cpu().numpy()
    ref = og.spmv(A, x)
    scale = _absrow(A, x)
    w = max(1, int(np.max(np.diff(A.rowptr))))
    assert np.all(np.abs(y64 - ref) <= (w + 1) * 2.0**-53 * scale + 1e-300)
    y32 = s.spmv(dev(x, torch.float32), "f32").cpu().numpy().astype(np.float64)
    assert np.all(np.abs(y32 - ref) <= (w + 3) * U32 * scale + 1e-30)
    s.close()


def test_spmv_f32_matches_oracle_f32_definition():
    """Same FP32 inputs on both sides: GPU FP32 SpMV vs the oracle's FP32 SpMV within the
    accumulation-order bound."""
    need_gpu()
    A = synth.convdiff2d(150, 4.0, 100.0)
    s = g.Solver(A, m=4)
    x32 = synth.uniform(A.n, 2).astype(np.float32)
    y = s.spmv(dev(x32, torch.float32), "f32").cpu().numpy()
    ref32 = og.spmv(A, x32, np.float32)
    scale = _absrow(A, x32.astype(np.float64))
    assert np.all(np.abs(y.astype(np.float64) - ref32) <= 10 * U32 * scale)
    s.close()


@pytest.mark.parametrize("k", [1, 7, 30])
def test_arnoldi_fp64_matches_oracle(k):
    need_gpu()
    A = synth.convdiff2d(60, 0.8, 100.0)          # n = 3600: 29 tiles, ragged tail
    r0 = synth.uniform(A.n, 5)
    s = g.Solver(A, m=40)
    H, V, steps = s.arnoldi(dev(r0), k, "f64")
    assert steps == k
    Vo, Ho, ko = og.arnoldi(A, r0, k)
    Anorm = np.linalg.norm(A.val)
    assert np.max(np.abs(H - Ho)) <= 1e-11 * Anorm
    V = V.cpu().numpy()
    assert np.max(np.abs(V - Vo)) <= 1e-10
    AV = np.column_stack([og.spmv(A, V[:, i]) for i in range(k)])
    assert np.linalg.norm(AV - V @ H) / Anorm <= 1e-13
    assert np.linalg.norm(np.eye(k + 1) - V.T @ V) <= 1e-13
    s.close()


@pytest.mark.parametrize("basis,orth_tol,h_tol", [("f32", 1e-5, 2e-5), ("bf16", 5e-2, 2e-2)])
def test_arnoldi_low_precision_bounds(basis, orth_tol, h_tol):
    need_gpu()
    A = synth.laplace3d(17)
    r0 = synth.uniform(A.n, 6)
    k = 25
    s = g.Solver(A, m=30, basis=basis)
    H, V, steps = s.arnoldi(dev(r0), k, "f32")
    assert steps == k
    Vo, Ho, _ = og.arnoldi(A, r0, k)
    Anorm = np.abs(A.val).max() * 7
    assert np.max(np.abs(H - Ho)) <= h_tol * Anorm
    V = V.cpu().numpy()
    assert np.linalg.norm(np.eye(k + 1) - V.T @ V) <= orth_tol * (k + 1)
    s.close()


def test_breakdown_on_eigenvector():
    need_gpu()
    # exact eigenvector of a diagonal matrix: the second basis vector is exactly zero
    d = np.linspace(1.0, 3.0, 300)
    A = synth.CSR(n=300, rowptr=np.arange(301, dtype=np.int32), colidx=np.arange(300, dtype=np.int32),
                  val=d)
    e = np.zeros(300)
    e[137] = 2.0
    s = g.Solver(A, m=10)
    H, V, steps = s.arnoldi(dev(e), 5, "f64")
    assert steps == 1 and H[0, 0] == d[137] and H[1, 0] == 0.0
    s.close()
    # a rounded Laplacian sine mode: Rayleigh quotient exact to rounding, tiny h_{2,1}
    N = 20
    A = synth.laplace2d(N)
    i = np.arange(1, N + 1)
    v = np.outer(np.sin(3 * np.pi * i / (N + 1)), np.sin(2 * np.pi * i / (N + 1))).ravel()
    s = g.Solver(A, m=10)
    H, V, steps = s.arnoldi(dev(v), 1, "f64")
    lam = (2 - 2 * np.cos(2 * np.pi / (N + 1))) + (2 - 2 * np.cos(3 * np.pi / (N + 1)))
    assert abs(H[0, 0] - lam) <= 1e-13 * lam and H[1, 0] <= 1e-13 * lam
    s.close()


@pytest.mark.parametrize("d", [3, 10, 25, 40])
def test_poly_roots_and_apply_match_oracle(d):
    need_gpu()
    A = synth.convdiff2d(97, 1.3, 100.0)
    start = synth.poly_start_vector(A.n, 0)
    s = g.Solver(A, m=30, poly_degree=d, poly_start=start)
    roots = s.poly_roots()
    P = og.poly_build(A, d, start)
    assert len(roots) == d + 1 == len(P.roots)
    # in Leja order, position by position (the order decides the FP32 stability of the product
    # form; the oracle's Leja scores are separated by >= 1e-3 here, far above the 1e-7 root noise)
    rg = np.asarray(roots)
    ro = np.asarray(P.roots)
    assert np.max(np.abs(rg - ro) / np.abs(ro)) <= 1e-7
    v = synth.uniform(A.n, 8)
    z64 = s.precond_apply(dev(v), "f64").cpu().numpy()
    zo = og.poly_apply(A, P, v)
    assert np.linalg.norm(z64 - zo) <= 1e-9 * np.linalg.norm(zo)
    z32 = s.precond_apply(dev(v, torch.float32), "f32").cpu().numpy().astype(np.float64)
    assert np.linalg.norm(z32 - zo) <= 1e-4 * np.linalg.norm(zo)
    s.close()


def _varied_rows(n, seed, long_rows=0, long_len=0):
    """Diagonally dominant nonsymmetric matrix whose rows hold 4-7 entries (plus `long_rows`
    rows of `long_len` entries)."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    longs = set(rng.choice(n, size=long_rows, replace=False).tolist()) if long_rows else set()
    for i in range(n):
        k = long_len if i in longs else int(rng.integers(4, 7))
        c = rng.choice(n, size=k, replace=False)
        c = c[c != i]
        v = rng.uniform(-0.5, 0.5, len(c)) * (4.0 / max(1, len(c)))
        rows += [i] * (len(c) + 1)
        cols += c.tolist() + [i]
        vals += v.tolist() + [8.0]
    order = np.argsort(np.array(rows), kind="stable")
    rows, cols, vals = np.array(rows)[order], np.array(cols)[order], np.array(vals)[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return synth.CSR(n=n, rowptr=np.cumsum(rp).astype(np.int32), colidx=cols.astype(np.int32),
                     val=vals)


@pytest.mark.parametrize("long_rows", [0, 12])
def test_fused_spmv_on_sliced_and_plain_rows(long_rows):
    """Rows of 4-7 entries take the sliced (SELL-32) copy in the fused SpMV + projection, with
    padded entries in most slices (the slices' widths add about a sixth to the nonzeros); twelve 400-entry rows make the padding exceed a quarter of the
    nonzeros, so the same kernel reads the CSR rows.  Both: the FP32 Arnoldi H against the
    oracle's FP64 one and the basis's orthogonality, and GMRES-IR against the oracle."""
    need_gpu()
    A = _varied_rows(20000, 5, long_rows, 400)
    b = synth.uniform(A.n, 8)
    s = g.Solver(A, m=30)
    k = 20
    H, V, steps = s.arnoldi(dev(b), k, "f32")
    assert steps == k
    Vo, Ho, _ = og.arnoldi(A, b, k)
    assert np.max(np.abs(H - Ho)) <= 2e-5 * 12.0
    V = V.cpu().numpy()
    assert np.linalg.norm(np.eye(k + 1) - V.T @ V) <= 1e-5 * (k + 1)
    x, st = s.ir_solve(dev(b), tol=1e-10)
    assert st.converged
    assert np.linalg.norm(b - og.spmv(A, x.cpu().numpy())) / np.linalg.norm(b) <= 1e-10
    ref = og.gmres_ir(A, b, m=30, tol=1e-10)
    assert abs(st.cycles - ref.cycles) <= 1
    s.close()
