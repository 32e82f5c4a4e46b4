"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module builds sparse matrices (CSR, int32 indices, float64 values) and right-hand sides.
It holds none of the solver's arithmetic: no matrix-vector products with the solver's data
flow, no Krylov steps, no preconditioner.  Everything is seeded with
``np.random.default_rng(seed)``.

Workloads (the paper's Galeri problems are not reproducible exactly, so these stand in):

* ``laplace2d(N)`` -- 5-point Laplacian on an N x N interior grid, Dirichlet boundary
  eliminated, lexicographic order (x fastest), unscaled stencil (4 on the diagonal, -1 off).
  nnz = 5 N^2 - 4 N.
* ``laplace3d(N)`` -- 7-point Laplacian on N^3 (6 / -1).  nnz = 7 N^3 - 6 N^2; N = 150 gives the
  paper's Laplace3D150 sizes n = 3,375,000, nnz = 23,490,000 (Section V, Table IV).
* ``convdiff2d(N, theta, peclet, shift)`` -- first-order upwind discretisation of
  -eps Lap u + (cos t, sin t) . grad u on the unit square, eps = 1/peclet, h = 1/(N+1),
  multiplied through by h^2/eps (beta = h * peclet): diagonal 4 + beta(|cos t| + |sin t|) + shift,
  upwind neighbour on each axis -1 - beta |component|, downwind neighbour -1.  Same sparsity as
  the paper's UniFlow2D2500 (n = 6,250,000, nnz = 31,240,000) for N = 2500.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """A square sparse matrix in CSR form with int32 indices and float64 values."""

    n: int
    rowptr: np.ndarray  # int32 [n+1]
    colidx: np.ndarray  # int32 [nnz], sorted within each row
    val: np.ndarray     # float64 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        """Dense copy (small matrices only); a plain scatter of the stored entries."""
        d = np.zeros((self.n, self.n))
        for i in range(self.n):
            for p in range(self.rowptr[i], self.rowptr[i + 1]):
                d[i, self.colidx[p]] += self.val[p]
        return d


def _assemble(n: int, cols: list[np.ndarray], vals: list[np.ndarray], masks: list[np.ndarray],
              name: str) -> CSR:
    """Assemble CSR from per-offset column/value/valid arrays given in increasing column order."""
    C = np.stack(cols, axis=1)
    V = np.stack(vals, axis=1)
    M = np.stack(masks, axis=1)
    counts = M.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = C[M].astype(np.int32)
    val = V[M].astype(np.float64)
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 index range")
    return CSR(n=n, rowptr=rowptr.astype(np.int32), colidx=colidx, val=val, name=name)


def laplace2d(N: int) -> CSR:
    """5-point Laplacian, 4 / -1, on an N x N grid (x fastest)."""
    n = N * N
    idx = np.arange(n, dtype=np.int64)
    ix, iy = idx % N, idx // N
    one = np.ones(n)
    cols = [idx - N, idx - 1, idx, idx + 1, idx + N]
    vals = [-one, -one, 4 * one, -one, -one]
    masks = [iy > 0, ix > 0, np.ones(n, bool), ix < N - 1, iy < N - 1]
    return _assemble(n, cols, vals, masks, f"laplace2d_{N}")


def laplace3d(N: int) -> CSR:
    """7-point Laplacian, 6 / -1, on an N x N x N grid (x fastest, then y, then z)."""
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    ix, iy, iz = idx % N, (idx // N) % N, idx // (N * N)
    one = np.ones(n)
    cols = [idx - N * N, idx - N, idx - 1, idx, idx + 1, idx + N, idx + N * N]
    vals = [-one, -one, -one, 6 * one, -one, -one, -one]
    masks = [iz > 0, iy > 0, ix > 0, np.ones(n, bool), ix < N - 1, iy < N - 1, iz < N - 1]
    return _assemble(n, cols, vals, masks, f"laplace3d_{N}")


def convdiff2d(N: int, theta: float, peclet: float = 100.0, shift: float = 0.0) -> CSR:
    """First-order upwind convection-diffusion on an N x N grid, wind (cos theta, sin theta)."""
    n = N * N
    h = 1.0 / (N + 1)
    beta = h * peclet
    cx, cy = np.cos(theta), np.sin(theta)
    idx = np.arange(n, dtype=np.int64)
    ix, iy = idx % N, idx // N
    one = np.ones(n)
    # west/east carry the x-upwind term, south/north the y-upwind term
    w_west = -1.0 - beta * abs(cx) if cx >= 0 else -1.0
    w_east = -1.0 if cx >= 0 else -1.0 - beta * abs(cx)
    w_south = -1.0 - beta * abs(cy) if cy >= 0 else -1.0
    w_north = -1.0 if cy >= 0 else -1.0 - beta * abs(cy)
    diag = 4.0 + beta * (abs(cx) + abs(cy)) + shift
    cols = [idx - N, idx - 1, idx, idx + 1, idx + N]
    vals = [w_south * one, w_west * one, diag * one, w_east * one, w_north * one]
    masks = [iy > 0, ix > 0, np.ones(n, bool), ix < N - 1, iy < N - 1]
    return _assemble(n, cols, vals, masks, f"convdiff2d_{N}")


def uniform(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform [lo, hi) float64 vector."""
    return np.random.default_rng(seed).uniform(lo, hi, n)


def dyadic_uniform01(n: int, seed: int, bits: int = 20) -> np.ndarray:
    """Uniform [0,1) quantised to multiples of 2^-bits, so that stencil products are exact."""
    u = np.random.default_rng(seed).uniform(0.0, 1.0, n)
    return np.floor(u * 2.0**bits) / 2.0**bits


def stencil_rhs_exact(A: CSR, xstar: np.ndarray, bits: int = 20) -> np.ndarray:
    """b = A x* for integer-valued A and dyadic x*, computed exactly in int64.

    Used only to build the right-hand side of the small Laplacian workload; the result carries
    no rounding, so every consumer sees the same b whatever its own arithmetic.
    """
    if not np.all(A.val == np.round(A.val)):
        raise ValueError("exact right-hand side needs integer matrix values")
    xi = np.round(xstar * 2.0**bits).astype(np.int64)
    vi = A.val.astype(np.int64)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    bi = np.zeros(A.n, dtype=np.int64)
    np.add.at(bi, rows, vi * xi[A.colidx])
    return bi.astype(np.float64) / 2.0**bits


# ---------------------------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------------------------

def workload_laplace2d_64():
    """2D 5-point Laplacian 64x64 (n = 4096), b = A x*, x* uniform[0,1) (dyadic) seed 0."""
    A = laplace2d(64)
    xstar = dyadic_uniform01(A.n, 0)
    return A, stencil_rhs_exact(A, xstar), xstar


def workload_laplace3d(N: int = 150, seed: int = 0):
    """3D 7-point Laplacian N^3 with b uniform[-1,1) seed `seed`."""
    A = laplace3d(N)
    return A, uniform(A.n, seed)


def workload_convdiff2d(N: int = 2500, seed: int = 0, peclet: float = 100.0):
    """2D upwind convection-diffusion N^2, theta ~ U[0, 2pi) and b ~ U[-1,1) from `seed`."""
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 2.0 * np.pi)
    A = convdiff2d(N, theta, peclet)
    return A, uniform(A.n, seed), theta


def poly_start_vector(n: int, seed: int = 0) -> np.ndarray:
    """Seeded U[-1,1) start vector of the polynomial preconditioner's Arnoldi process."""
    return uniform(n, seed)


def workload_batched(nsys: int = 256, nrhs: int = 8, side_lo: int = 32, side_hi: int = 320,
                     peclet: float = 100.0, seed0: int = 0):
    """Many independent convection-diffusion systems of uneven size (the batched workload).

    System s draws from ``default_rng(seed0 + s)``: the grid side N ~ U{side_lo..side_hi}, the
    wind angle theta ~ U[0, 2 pi), a diagonal shift sigma ~ U[0, 0.5], and nrhs right-hand sides
    ~ U[-1, 1) (an n x nrhs array).  Returns a list of (CSR, B).
    """
    out = []
    for s in range(nsys):
        rng = np.random.default_rng(seed0 + s)
        N = int(rng.integers(side_lo, side_hi + 1))
        theta = rng.uniform(0.0, 2.0 * np.pi)
        sigma = rng.uniform(0.0, 0.5)
        A = convdiff2d(N, theta, peclet, sigma)
        A.name = f"batch{seed0 + s}_conv{N}"
        out.append((A, rng.uniform(-1.0, 1.0, (A.n, nrhs))))
    return out


def workload_controller(index: int, side_lo: int = 64, side_hi: int = 256):
    """One system of the parameter-controller population (training and held-out sets).

    System ``index`` draws from ``default_rng(10_000 + index)``: the grid side N ~ U{side_lo..side_hi},
    the Peclet number log-uniform on [1, 1000], the wind angle theta ~ U[0, 2 pi) and b ~ U[-1, 1).
    The polynomial start vector is ``poly_start_vector(n)``.  Returns (CSR, b, start).
    """
    rng = np.random.default_rng(10_000 + index)
    N = int(rng.integers(side_lo, side_hi + 1))
    peclet = float(10.0 ** rng.uniform(0.0, 3.0))
    theta = rng.uniform(0.0, 2.0 * np.pi)
    A = convdiff2d(N, theta, peclet)
    A.name = f"ctrl{index}_conv{N}_pe{peclet:.0f}"
    return A, rng.uniform(-1.0, 1.0, A.n), poly_start_vector(A.n)


def _from_coo(n: int, rows, cols, vals, name: str) -> CSR:
    """CSR from coordinate triplets without duplicates, columns sorted within each row."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], np.asarray(vals, dtype=np.float64)[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n=n, rowptr=rowptr.astype(np.int32), colidx=cols.astype(np.int32), val=vals,
               name=name)


def aniso2d(N: int, eps: float) -> CSR:
    """-u_xx - eps u_yy on an N x N grid (5-point, unscaled: diagonal 2 + 2 eps, x neighbours -1,
    y neighbours -eps): strongly coupled along x when eps << 1."""
    n = N * N
    idx = np.arange(n).reshape(N, N)            # idx[y, x]
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [np.full(n, 2.0 + 2.0 * eps)]
    for dy, dx, w in ((0, 1, -1.0), (0, -1, -1.0), (1, 0, -eps), (-1, 0, -eps)):
        ys, xs = np.nonzero(np.ones((N, N), bool))
        ny, nx = ys + dy, xs + dx
        ok = (ny >= 0) & (ny < N) & (nx >= 0) & (nx < N)
        rows.append(idx[ys[ok], xs[ok]])
        cols.append(idx[ny[ok], nx[ok]])
        vals.append(np.full(ok.sum(), w))
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                     f"aniso2d_{N}_eps{eps:g}")


def permute_symmetric(A: CSR, seed: int) -> CSR:
    """P A P^T for a seeded random relabelling of the unknowns (destroys the natural ordering)."""
    rng = np.random.default_rng(seed)
    p = rng.permutation(A.n)                      # new label of old node i is p[i]
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return _from_coo(A.n, p[rows], p[np.asarray(A.colidx)], A.val, A.name + f"_perm{seed}")


def hetero2d(N: int, contrast: float = 1e4, seed: int = 0) -> CSR:
    """-div(k grad u) on an N x N grid with a seeded log-uniform nodal coefficient k in
    [1, contrast] (5-point: the coupling of neighbours i, j is the harmonic mean 2 k_i k_j /
    (k_i + k_j); Dirichlet boundary edges weigh k_i).  Symmetric positive definite, with row
    scales spread over `contrast`."""
    rng = np.random.default_rng(seed)
    n = N * N
    k = np.exp(rng.uniform(0.0, np.log(contrast), n))
    idx = np.arange(n).reshape(N, N)
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        ys, xs = np.nonzero(np.ones((N, N), bool))
        ny, nx = ys + dy, xs + dx
        inside = (ny >= 0) & (ny < N) & (nx >= 0) & (nx < N)
        i = idx[ys, xs]
        j = np.where(inside, idx[np.clip(ny, 0, N - 1), np.clip(nx, 0, N - 1)], 0)
        w = np.where(inside, 2.0 * k[i] * k[j] / (k[i] + k[j]), k[i])
        np.add.at(diag, i, w)
        rows.append(i[inside])
        cols.append(j[inside])
        vals.append(-w[inside])
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                     f"hetero2d_{N}_c{contrast:g}")


def random_rows(n: int, per_row: int, band: int, seed: int = 0) -> CSR:
    """A nonsymmetric matrix with long rows: row i holds the diagonal and `per_row - 1` distinct
    seeded random columns within |j - i| <= band (values U[-1, 1)), and a diagonal of
    1.2 x (the row's off-diagonal absolute sum), so it is strictly diagonally dominant.  Rows
    near the edges keep the columns that fall inside [0, n) (so row lengths vary)."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i0 in range(0, n, 4096):
        i = np.arange(i0, min(n, i0 + 4096))
        off = rng.integers(-band, band + 1, size=(i.size, 3 * per_row))
        off[off >= 0] += 1                                 # no zero offset: the diagonal is apart
        for r, o in zip(i, off):
            c = np.unique(r + o)
            c = c[(c >= 0) & (c < n)][: per_row - 1]
            v = rng.uniform(-1.0, 1.0, c.size)
            rows.append(np.full(c.size + 1, r))
            cols.append(np.concatenate([c, [r]]))
            vals.append(np.concatenate([v, [1.2 * np.abs(v).sum() + 1e-3]]))
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                     f"random_rows_{n}_{per_row}_b{band}_s{seed}")
