"""Pins of the CPU oracle against what the mathematics fixes (no GPU).

Every test here checks the oracle against something other than itself: closed-form eigenpairs
of the Laplacians, direct dense solves, the Arnoldi relation, exact termination on matrices with
k distinct eigenvalues, the Givens least-squares solution against a library least-squares solve,
and the defining optimality property of the GMRES polynomial.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import gmres as og


def _sine_mode_2d(N, kx, ky):
    i = np.arange(1, N + 1)
    sx = np.sin(kx * np.pi * i / (N + 1))
    sy = np.sin(ky * np.pi * i / (N + 1))
    v = np.outer(sy, sx).ravel()          # x fastest
    lam = (2 - 2 * np.cos(kx * np.pi / (N + 1))) + (2 - 2 * np.cos(ky * np.pi / (N + 1)))
    return v, lam


def _sine_mode_3d(N, kx, ky, kz):
    i = np.arange(1, N + 1)
    s = [np.sin(k * np.pi * i / (N + 1)) for k in (kx, ky, kz)]
    v = np.einsum("z,y,x->zyx", s[2], s[1], s[0]).ravel()
    lam = sum(2 - 2 * np.cos(k * np.pi / (N + 1)) for k in (kx, ky, kz))
    return v, lam


def _diag_csr(d):
    n = len(d)
    return synth.CSR(n=n, rowptr=np.arange(n + 1, dtype=np.int32),
                     colidx=np.arange(n, dtype=np.int32), val=np.asarray(d, float))


def _dense_csr(M):
    n = M.shape[0]
    rows, cols = np.nonzero(M)
    rowptr = np.zeros(n + 1, np.int32)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    return synth.CSR(n=n, rowptr=rowptr, colidx=cols.astype(np.int32), val=M[rows, cols])


# --------------------------------------------------------------------------- SpMV

@pytest.mark.parametrize("N,k", [(16, (1, 1)), (16, (3, 7)), (33, (5, 2))])
def test_spmv_laplace2d_sine_modes(N, k):
    A = synth.laplace2d(N)
    v, lam = _sine_mode_2d(N, *k)
    y = og.spmv(A, v)
    assert np.linalg.norm(y - lam * v) <= 1e-13 * lam * np.linalg.norm(v) * 10


@pytest.mark.parametrize("N,k", [(9, (1, 1, 1)), (12, (2, 5, 3))])
def test_spmv_laplace3d_sine_modes(N, k):
    A = synth.laplace3d(N)
    v, lam = _sine_mode_3d(N, *k)
    y = og.spmv(A, v)
    assert np.linalg.norm(y - lam * v) <= 1e-13 * lam * np.linalg.norm(v) * 10


def test_laplace_sizes_match_paper():
    # Laplace3D150: n = 3,375,000 and nnz = 23,490,000 (Table IV); 2D N=2500: 31,240,000 (Table IV)
    N = 150
    assert N**3 == 3_375_000 and 7 * N**3 - 6 * N**2 == 23_490_000
    N = 2500
    assert N * N == 6_250_000 and 5 * N * N - 4 * N == 31_240_000
    A = synth.laplace3d(20)
    assert A.nnz == 7 * 20**3 - 6 * 20**2
    C = synth.convdiff2d(30, 1.0)
    assert C.nnz == 5 * 30 * 30 - 4 * 30


def test_spmv_convdiff_against_stencil_formula():
    """Dense operator written point by point from the upwind stencil, applied by dense matmul."""
    N, theta, pe, shift = 6, 2.4, 100.0, 0.3
    A = synth.convdiff2d(N, theta, pe, shift)
    h = 1.0 / (N + 1)
    beta = h * pe
    cx, cy = np.cos(theta), np.sin(theta)
    D = np.zeros((N * N, N * N))
    for iy in range(N):
        for ix in range(N):
            r = iy * N + ix
            D[r, r] = 4 + beta * (abs(cx) + abs(cy)) + shift
            nb = {(-1, 0): -1 - (beta * abs(cx) if cx >= 0 else 0),
                  (1, 0): -1 - (beta * abs(cx) if cx < 0 else 0),
                  (0, -1): -1 - (beta * abs(cy) if cy >= 0 else 0),
                  (0, 1): -1 - (beta * abs(cy) if cy < 0 else 0)}
            for (dx, dy), c in nb.items():
                jx, jy = ix + dx, iy + dy
                if 0 <= jx < N and 0 <= jy < N:
                    D[r, jy * N + jx] = c
    x = np.random.default_rng(3).standard_normal(N * N)
    assert np.allclose(og.spmv(A, x), D @ x, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------- bfloat16 rounding

def test_round_bf16_ties_and_library():
    one = np.float32(1.0)
    ulp = 2.0**-7
    vals = np.array([1.0, 1 + ulp / 2, 1 + 1.5 * ulp, 1 + ulp / 2 + 2**-20, -3.14159, 1e-30, 6e4],
                    dtype=np.float32)
    got = og.round_bf16(vals)
    assert got[0] == one and got[1] == one               # tie to even (down)
    assert got[2] == np.float32(1 + 2 * ulp)             # tie to even (up)
    assert got[3] == np.float32(1 + ulp)                 # above the tie
    ref = torch.from_numpy(vals).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(got, ref)
    r = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 1e3
    assert np.array_equal(og.round_bf16(r),
                          torch.from_numpy(r).to(torch.bfloat16).to(torch.float32).numpy())


# --------------------------------------------------------------------------- Arnoldi / CGS2

def test_arnoldi_relation_and_orthogonality():
    A = synth.convdiff2d(16, 0.7, 100.0)
    v0 = synth.uniform(A.n, 1)
    V, H, k = og.arnoldi(A, v0, 30)
    assert k == 30 and V.shape == (A.n, 31) and H.shape == (31, 30)
    AV = np.column_stack([og.spmv(A, V[:, i]) for i in range(k)])
    Anorm = np.linalg.norm(A.val)
    assert np.linalg.norm(AV - V @ H) / Anorm <= 1e-13
    assert np.linalg.norm(np.eye(k + 1) - V.T @ V) <= 1e-13
    assert np.allclose(np.tril(H, -2), 0)                 # upper Hessenberg
    assert np.all(np.diag(H, -1) > 0)


def test_givens_matches_library_lstsq():
    rng = np.random.default_rng(5)
    for k in (1, 2, 7, 40):
        H = np.triu(rng.standard_normal((k + 1, k)), -1)
        y, res = og.lstsq_givens(H, 2.5)
        rhs = np.zeros(k + 1)
        rhs[0] = 2.5
        yl, *_ = np.linalg.lstsq(H, rhs, rcond=None)
        assert np.allclose(y, yl, rtol=1e-10, atol=1e-12)
        assert abs(res - np.linalg.norm(rhs - H @ yl)) <= 1e-12 * 2.5


def test_implicit_equals_explicit_each_step():
    A = synth.convdiff2d(20, 4.0, 50.0)
    b = synth.uniform(A.n, 2)
    cyc = og.gmres_cycle(lambda z: og.spmv(A, z), b, 40)
    for j in range(1, cyc.k + 1):
        y, _ = og.lstsq_givens(cyc.H[: j + 1, :j], cyc.gamma)
        x = cyc.V[:, :j] @ y
        explicit = np.linalg.norm(b - og.spmv(A, x))
        assert abs(explicit - cyc.implicit[j - 1]) <= 1e-12 * cyc.gamma


# --------------------------------------------------------------------------- GMRES solves

def test_full_krylov_equals_direct_solve():
    rng = np.random.default_rng(11)
    n = 60
    M = rng.standard_normal((n, n)) + n * np.eye(n) * 0.3
    A = _dense_csr(M)
    b = rng.standard_normal(n)
    res = og.gmres(A, b, m=n, tol=1e-14)
    xd = np.linalg.solve(M, b)
    kappa = np.linalg.cond(M)
    assert np.linalg.norm(res.x - xd) / np.linalg.norm(xd) <= kappa * 1e-13
    assert res.cycles == 1


def _lu_solve(M, b):
    """Dense Gaussian elimination with partial pivoting, written out (no LAPACK)."""
    A = np.array(M, dtype=np.float64)
    x = np.array(b, dtype=np.float64)
    n = A.shape[0]
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if p != k:
            A[[k, p]] = A[[p, k]]
            x[[k, p]] = x[[p, k]]
        for i in range(k + 1, n):
            f = A[i, k] / A[k, k]
            A[i, k:] -= f * A[k, k:]
            x[i] -= f * x[k]
    for i in range(n - 1, -1, -1):
        x[i] = (x[i] - A[i, i + 1:] @ x[i + 1:]) / A[i, i]
    return x


@pytest.mark.parametrize("n,seed", [(40, 3), (120, 4), (200, 5)])
def test_gmres_full_space_matches_own_lu_on_nonsymmetric_dominant_systems(n, seed):
    """GMRES(m >= n) in FP64 solves a random nonsymmetric, diagonally dominant system to the
    accuracy of a partial-pivot LU solve: relative difference <= kappa * 1e-12."""
    rng = np.random.default_rng(seed)
    M = rng.uniform(-1.0, 1.0, (n, n))
    M += np.diag(np.abs(M).sum(axis=1) * rng.uniform(1.05, 1.5, n))
    b = rng.uniform(-1.0, 1.0, n)
    xl = _lu_solve(M, b)
    assert np.linalg.norm(M @ xl - b) <= 1e-13 * np.linalg.norm(b) * n
    res = og.gmres(_dense_csr(M), b, m=n, tol=1e-14)
    kappa = np.linalg.cond(M)
    assert res.converged
    assert np.linalg.norm(res.x - xl) / np.linalg.norm(xl) <= kappa * 1e-12


def test_k_distinct_eigenvalues_terminate_in_k_steps():
    lam = np.array([0.5, 1.0, 2.0, 3.5, 5.0, 8.0, 13.0])
    d = np.repeat(lam, 10)
    A = _diag_csr(d)
    b = synth.uniform(A.n, 4)
    cyc = og.gmres_cycle(lambda z: og.spmv(A, z), b, 50, stop_abs=1e-12 * np.linalg.norm(b))
    assert cyc.k == len(lam)
    assert cyc.implicit[-2] > 1e-3 * np.linalg.norm(b)      # not converged one step earlier
    x = cyc.V[:, : cyc.k] @ cyc.y
    assert np.linalg.norm(x - b / d) / np.linalg.norm(b / d) <= 1e-12


def test_exact_lucky_breakdown():
    d = np.array([2.0, 3.0, 5.0, 7.0])
    A = _diag_csr(d)
    b = np.array([0.0, 0.0, 4.0, 0.0])           # an eigenvector: A b = 5 b exactly
    cyc = og.gmres_cycle(lambda z: og.spmv(A, z), b, 3)
    assert cyc.breakdown and cyc.k == 1
    assert np.allclose(cyc.V[:, :1] @ cyc.y, b / d, atol=1e-15)


def test_eigenvector_rhs_converges_in_one_step():
    A = synth.laplace2d(20)
    v, lam = _sine_mode_2d(20, 2, 3)
    res = og.gmres(A, v, m=50, tol=1e-12)
    assert res.iters == 1
    assert np.allclose(res.x, v / lam, rtol=0, atol=1e-12)


def test_laplace2d_64_solution_error_within_condition_bound():
    A, b, xstar = synth.workload_laplace2d_64()
    N = 64
    lmin = 2 * (2 - 2 * np.cos(np.pi / (N + 1)))
    lmax = 2 * (2 - 2 * np.cos(N * np.pi / (N + 1)))
    kappa = lmax / lmin
    res = og.gmres(A, b, m=50, tol=1e-10)
    assert res.converged and res.rel_res <= 1e-10
    assert np.linalg.norm(res.x - xstar) / np.linalg.norm(xstar) <= kappa * 1e-10
    # the implicit residual at the stop agrees with the explicit one
    assert res.loss_of_accuracy == 0


def test_gmres_ir_converges_and_tracks_fp64():
    A, b, xstar = synth.workload_laplace2d_64()
    r64 = og.gmres(A, b, m=50, tol=1e-10)
    rir = og.gmres_ir(A, b, m=50, tol=1e-10)
    assert rir.converged and rir.rel_res <= 1e-10
    assert rir.iters % 50 == 0                                # full inner cycles (Section III-B)
    assert rir.cycles <= r64.cycles + 2                       # IR tracks FP64 (Section V-B)
    assert np.linalg.norm(rir.x - r64.x) / np.linalg.norm(r64.x) <= 1e-7


def test_gmres_ir_bf16_basis_still_reaches_fp64_accuracy():
    A = synth.convdiff2d(48, 1.1, 100.0)
    b = synth.uniform(A.n, 0)
    rir = og.gmres_ir(A, b, m=30, tol=1e-10, basis="bf16")
    assert rir.converged and rir.rel_res <= 1e-10


def test_fp32_only_gmres_stalls_above_double_accuracy():
    # Section V-B: single precision GMRES alone levels off far above 1e-10
    A = synth.convdiff2d(48, 1.1, 100.0)
    b = synth.uniform(A.n, 0)
    res = og.gmres(A, b, m=50, tol=1e-10, dtype=np.float32, maxiter=4000, max_loa=10**9)
    assert not res.converged
    assert min(res.history) > 1e-9


# --------------------------------------------------------------------------- polynomial

def test_poly_on_diagonal_is_exact_inverse():
    lam = np.array([0.7, 1.3, 2.0, 2.9, 4.1, 6.0])
    A = _diag_csr(lam)
    v0 = np.array([1.0, -0.5, 0.25, 0.8, -0.9, 0.6])
    P = og.poly_build(A, len(lam) - 1, v0)
    assert P.degree == len(lam) - 1
    assert np.allclose(np.sort(P.roots.real), lam, rtol=1e-10)
    x = synth.uniform(A.n, 9)
    z = og.poly_apply(A, P, x)
    assert np.allclose(lam * z, x, rtol=1e-10, atol=1e-12)


def test_poly_degree_drops_at_breakdown():
    lam = np.repeat(np.array([1.0, 2.0, 3.0]), 4)
    A = _diag_csr(lam)
    P = og.poly_build(A, 6, synth.uniform(A.n, 1) + 2.0)
    assert P.degree == 2
    x = synth.uniform(A.n, 2)
    assert np.allclose(lam * og.poly_apply(A, P, x), x, rtol=1e-10)


@pytest.mark.parametrize("d", [1, 3, 5, 8])
def test_poly_application_equals_gmres_iterate(d):
    """The GMRES polynomial is the one GMRES itself applies: after d+1 unrestarted steps from
    x0 = 0 on A x = v, the iterate is p(A) v and the residual pi(A) v."""
    A = synth.convdiff2d(12, 2.2, 30.0)
    v = synth.uniform(A.n, 7)
    P = og.poly_build(A, d, v)
    cyc = og.gmres_cycle(lambda z: og.spmv(A, z), v, d + 1)
    xg = cyc.V[:, : cyc.k] @ cyc.y
    z = og.poly_apply(A, P, v)
    assert np.linalg.norm(z - xg) <= 1e-8 * np.linalg.norm(xg)


def test_poly_degree1_closed_form():
    """Degree 1: p(t) = c0 + c1 t minimises ||v - A (c0 v + c1 A v)||, a 2-column least squares."""
    A = synth.convdiff2d(10, 0.4, 10.0)
    v = synth.uniform(A.n, 3)
    P = og.poly_build(A, 1, v)
    Av = og.spmv(A, v)
    AAv = og.spmv(A, Av)
    c, *_ = np.linalg.lstsq(np.column_stack([Av, AAv]), v, rcond=None)
    assert np.allclose(og.poly_power_coeffs(P), c, rtol=1e-9)


@pytest.mark.parametrize("d", [2, 4, 6])
def test_poly_product_and_power_forms_agree(d):
    A = synth.laplace2d(10)
    v = synth.uniform(A.n, 5)
    P = og.poly_build(A, d, synth.uniform(A.n, 6))
    z1 = og.poly_apply(A, P, v)
    z2 = og.poly_apply_power(A, og.poly_power_coeffs(P), v)
    assert np.linalg.norm(z1 - z2) <= 1e-9 * np.linalg.norm(z1)


def test_leja_order_properties():
    th = np.array([1.0, 3 + 2j, 3 - 2j, 0.2, 5.0, 2 - 0.5j, 2 + 0.5j])
    o = og.leja_order(th)
    assert len(o) == len(th)
    assert abs(o[0]) == max(abs(th))
    for i, t in enumerate(o):
        if t.imag > 0:
            assert o[i + 1] == np.conj(t)
    assert sorted(np.round(o, 12), key=lambda z: (z.real, z.imag)) == \
        sorted(np.round(th, 12), key=lambda z: (z.real, z.imag))


def test_leja_order_hand_worked_example():
    """A six-value set ordered by hand (tests/golden/leja_hand_example.json, integer squared
    distances, every comparison exact): the product rule's order, which a sum of distances or a
    largest-smallest-distance rule would not give."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "leja_hand_example.json")))
    th = np.array(gold["theta_re"]) + 1j * np.array(gold["theta_im"])
    want = np.array(gold["expected_re"]) + 1j * np.array(gold["expected_im"])
    assert np.array_equal(og.leja_order(th), want)
    # the order does not depend on the order the values come in
    perm = np.random.default_rng(3).permutation(len(th))
    assert np.array_equal(og.leja_order(th[perm]), want)


def _leja_defining_property(theta, order):
    """Check an ordering against the modified Leja rule written out directly: the first pick has
    the largest modulus; every later pick (a real value, or a complex value with Im > 0 followed
    at once by its conjugate) has a product of distances to all values placed before it at least
    as large as that of every value not yet placed.  Products are formed as plain products."""
    assert len(order) == len(theta)
    placed = []
    rest = [complex(t) for t in theta]
    i = 0
    while i < len(order):
        z = complex(order[i])
        if not placed:
            assert abs(z) >= max(abs(c) for c in rest) * (1 - 1e-14)
        else:
            pz = np.prod([abs(z - c) for c in placed])
            for c in rest:
                assert pz >= np.prod([abs(c - q) for q in placed]) * (1 - 1e-12)
        k = int(np.argmin([abs(c - z) for c in rest]))
        assert abs(rest[k] - z) <= 1e-14 * max(1.0, abs(z))
        rest.pop(k)
        placed.append(z)
        if z.imag != 0.0:
            assert z.imag > 0 and complex(order[i + 1]) == z.conjugate()
            k = int(np.argmin([abs(c - z.conjugate()) for c in rest]))
            rest.pop(k)
            placed.append(z.conjugate())
            i += 2
        else:
            i += 1
    assert not rest


@pytest.mark.parametrize("seed", range(12))
def test_leja_order_meets_its_defining_rule_on_random_sets(seed):
    """Brute-force check of every pick on random sets of real values and conjugate pairs."""
    rng = np.random.default_rng(seed)
    nr, nc = int(rng.integers(0, 6)), int(rng.integers(0, 4))
    re = list(rng.uniform(-3, 3, nr))
    for _ in range(nc):
        a, b = rng.uniform(-3, 3), rng.uniform(0.1, 2)
        re += [complex(a, b), complex(a, -b)]
    th = np.array(re, dtype=complex)
    th = th[rng.permutation(len(th))]
    if len(th) == 0:
        return
    _leja_defining_property(th, og.leja_order(th))


def test_leja_order_of_a_degree_25_polynomial_meets_its_rule():
    A = synth.convdiff2d(60, 0.4, 100.0)
    P = og.poly_build(A, 25, synth.poly_start_vector(A.n, 0))
    _leja_defining_property(P.roots, P.roots)


def test_preconditioned_gmres_converges_faster():
    A = synth.convdiff2d(40, 0.9, 100.0)
    b = synth.uniform(A.n, 0)
    P = og.poly_build(A, 10, synth.poly_start_vector(A.n, 0))
    r0 = og.gmres(A, b, m=30, tol=1e-10)
    rp = og.gmres(A, b, m=30, tol=1e-10, poly=P)
    assert rp.converged and r0.converged
    assert rp.iters * 4 < r0.iters
    rir = og.gmres_ir(A, b, m=30, tol=1e-10, poly=P)
    assert rir.converged and rir.rel_res <= 1e-10


def test_fp64_gmres_with_fp32_polynomial_reaches_fp64_accuracy():
    """variant (a) of Section III-D: an FP32 polynomial inside FP64 GMRES still reaches a 1e-10
    residual, at the price of at most one extra restart here: the FP32 operator is not exactly
    the linear map GMRES assumes, so the implicit residual can run ahead of the explicit one
    (the loss of accuracy of Section V-F).  The FP32 application differs from the FP64 one by a
    rounding-level relative amount."""
    A = synth.convdiff2d(48, 0.7, peclet=100.0)
    b = synth.uniform(A.n, 3)
    poly = og.poly_build(A, 10, synth.poly_start_vector(A.n))
    r64 = og.gmres(A, b, 30, 1e-10, poly=poly)
    r32 = og.gmres(A, b, 30, 1e-10, poly=poly, poly_dtype=np.float32)
    assert r64.converged and r32.converged
    assert r32.rel_res <= 1e-10
    assert r64.loss_of_accuracy == 0
    assert r64.iters <= r32.iters <= r64.iters + 30
    v = synth.uniform(A.n, 5)
    z64 = og.poly_apply(A, poly, v)
    z32 = og.poly_apply(A, poly, v.astype(np.float32), np.float32).astype(np.float64)
    assert np.linalg.norm(z32 - z64) <= 1e-5 * np.linalg.norm(z64)
    assert np.linalg.norm(z32 - z64) > 0.0


def test_poly_dtype_default_is_the_solve_precision():
    A = synth.laplace2d(20)
    b = synth.uniform(A.n, 1)
    poly = og.poly_build(A, 5, synth.poly_start_vector(A.n))
    a = og.gmres(A, b, 20, 1e-10, poly=poly)
    c = og.gmres(A, b, 20, 1e-10, poly=poly, poly_dtype=np.float64)
    np.testing.assert_array_equal(a.x, c.x)


def test_gmres_fd_switch_zero_is_fp64_gmres_and_any_switch_converges():
    A = synth.convdiff2d(40, 0.3, peclet=50.0)
    b = synth.uniform(A.n, 2)
    ref = og.gmres(A, b, 25, 1e-10)
    r0, k0 = og.gmres_fd(A, b, 25, 1e-10, 0)
    assert k0 == 0 and r0.iters == ref.iters
    np.testing.assert_array_equal(r0.x, ref.x)
    for sw in (25, 100, 400):
        r, k = og.gmres_fd(A, b, 25, 1e-10, sw)
        assert r.converged and r.rel_res <= 1e-10
        assert k == min(sw, k)            # the FP32 phase stops at the switch point
        assert k <= sw and r.iters >= k
        # the FP32 phase's residuals are those of single-precision GMRES on its own
        r32 = og.gmres(A, b, 25, 1e-10, maxiter=sw, dtype=np.float32, max_loa=1 << 30)
        assert r.history[: len(r32.history)] == r32.history


def test_fp32_phase_stalls_where_fp64_continues():
    """Single-precision GMRES stalls near FP32 accuracy; the FP64 phase carries on from its
    iterate (Section V-A's premise)."""
    A = synth.laplace2d(40)
    b = synth.uniform(A.n, 4)
    r32 = og.gmres(A, b, 30, 1e-10, maxiter=3000, dtype=np.float32, max_loa=1 << 30)
    assert not r32.converged and 1e-8 < r32.rel_res < 1e-4
    r, k = og.gmres_fd(A, b, 30, 1e-10, 3000)
    assert r.converged and k == r32.iters


def test_round_f16_scaled_keeps_relative_precision_where_raw_fp16_does_not():
    n = 4_000_000
    rng = np.random.default_rng(0)
    v = rng.standard_normal(n).astype(np.float32)
    v /= np.linalg.norm(v)                          # unit vector: entries ~ 5e-4, many far smaller
    q = og.round_f16_scaled(v)
    rel = np.abs(q - v) / np.maximum(np.abs(v), 1e-30)
    big = np.abs(v) * np.sqrt(n) > 2.0 ** -14       # scaled entries in FP16's normal range
    assert rel[big].max() <= 2.0 ** -11 * 1.0001    # half an ulp of FP16 (plus the FP32 division)
    raw = v.astype(np.float16).astype(np.float32)   # unscaled: the small entries go subnormal
    rel_raw = np.abs(raw - v) / np.maximum(np.abs(v), 1e-30)
    small = (np.abs(v) < 2.0 ** -15) & big           # subnormal in raw FP16, normal when scaled
    assert small.sum() > 1000
    assert np.median(rel_raw[small]) > 4 * np.median(rel[small])
    # values on the scaled FP16 grid are kept exactly
    g = (np.arange(-100, 100, dtype=np.float32) / 64).astype(np.float16).astype(np.float32)
    w = g / np.float32(np.sqrt(g.shape[0]))
    np.testing.assert_allclose(og.round_f16_scaled(w), w, rtol=1e-7, atol=0)


def test_gmres_ir_f16_basis_reaches_fp64_accuracy():
    A = synth.laplace2d(48)
    b = synth.uniform(A.n, 5)
    r32 = og.gmres_ir(A, b, 40, 1e-10)
    r16 = og.gmres_ir(A, b, 40, 1e-10, basis="f16")
    assert r16.converged and r16.rel_res <= 1e-10
    assert r16.cycles <= r32.cycles + 2


# ---------------------------------------------------------------- delayed CGS2 (DCGS2) variant

def test_dcgs2_equals_cgs2_in_fp64():
    """DCGS2 and CGS2 build the same Arnoldi factorisation in exact arithmetic (it is unique for
    an unreduced Hessenberg matrix and a given start vector): in FP64 their H, V and y agree to
    rounding.  A wrong coefficient, sign or index in the delayed pass breaks the equality."""
    A = synth.convdiff2d(30, 0.7, 100.0)
    r0 = synth.uniform(A.n, 1)
    op = lambda z: og.spmv(A, z)
    for m in (1, 2, 7, 25):
        c1 = og.gmres_cycle(op, r0, m)
        c2 = og.gmres_cycle_dcgs2(op, r0, m)
        assert c1.k == c2.k == m
        assert np.max(np.abs(c1.H - c2.H)) <= 1e-13 * np.max(np.abs(c1.H))
        assert np.max(np.abs(c1.V[:, :m + 1] - c2.V[:, :m + 1])) <= 1e-13
        assert np.max(np.abs(c1.y - c2.y)) <= 1e-12 * np.max(np.abs(c1.y))
        assert np.allclose(c1.implicit, c2.implicit, rtol=1e-12, atol=0)


def test_dcgs2_arnoldi_relation_and_orthogonality():
    A = synth.laplace2d(24)
    r0 = synth.uniform(A.n, 4)
    op = lambda z: og.spmv(A, z)
    c = og.gmres_cycle_dcgs2(op, r0, 40)
    V, H, k = c.V, c.H, c.k
    AV = np.column_stack([op(V[:, i]) for i in range(k)])
    assert np.linalg.norm(AV - V @ H) <= 1e-13 * 8.0 * np.sqrt(k)          # ||A||_2 <= 8
    assert np.linalg.norm(np.eye(k + 1) - V.T @ V) <= 1e-13


def test_dcgs2_terminates_in_k_steps_on_k_distinct_eigenvalues():
    lam = np.array([0.5, 1.0, 2.0, 3.5, 5.0, 8.0, 13.0])
    d = np.repeat(lam, 10)
    A = _diag_csr(d)
    b = synth.uniform(A.n, 4)
    cyc = og.gmres_cycle_dcgs2(lambda z: og.spmv(A, z), b, 50, stop_abs=1e-12 * np.linalg.norm(b))
    assert cyc.k == len(lam)
    assert cyc.implicit[-2] > 1e-3 * np.linalg.norm(b)      # not converged one step earlier
    x = cyc.V[:, : cyc.k] @ cyc.y
    assert np.linalg.norm(x - b / d) / np.linalg.norm(b / d) <= 1e-12


def test_dcgs2_exact_lucky_breakdown():
    d = np.array([2.0, 3.0, 5.0, 7.0])
    A = _diag_csr(d)
    b = np.array([0.0, 0.0, 4.0, 0.0])           # an eigenvector: A b = 5 b exactly
    cyc = og.gmres_cycle_dcgs2(lambda z: og.spmv(A, z), b, 3)
    assert cyc.breakdown and cyc.k == 1
    assert np.allclose(cyc.V[:, :1] @ cyc.y, b / d, atol=1e-15)


def test_dcgs2_full_space_gmres_equals_a_direct_solve():
    rng = np.random.default_rng(11)
    n = 60
    M = rng.standard_normal((n, n)) + 0.5 * n * np.eye(n)
    A = _dense_csr(M)
    b = rng.standard_normal(n)
    r = og.gmres(A, b, n, 1e-13, orth="dcgs2")
    x = np.linalg.solve(M, b)
    assert r.converged and np.linalg.norm(r.x - x) <= np.linalg.cond(M) * 1e-13 * np.linalg.norm(x)


def test_dcgs2_eigenvector_rhs_converges_in_one_step():
    A = synth.laplace2d(20)
    v, lam = _sine_mode_2d(20, 2, 3)
    res = og.gmres(A, v, m=50, tol=1e-12, orth="dcgs2")
    assert res.iters == 1
    assert np.allclose(res.x, v / lam, rtol=0, atol=1e-12)


@pytest.mark.parametrize("basis", ["f32", "bf16"])
def test_dcgs2_fp32_cycle_orthogonality_and_ir_accuracy(basis):
    A = synth.convdiff2d(40, 1.1, 100.0)
    b = synth.uniform(A.n, 6)
    rnd = og.round_bf16 if basis == "bf16" else None
    c = og.gmres_cycle_dcgs2(lambda z: og.spmv(A, z, np.float32), b.astype(np.float32), 30,
                             dtype=np.float32, basis_round=rnd)
    V = c.V[:, : c.k].astype(np.float64)
    bound = 1e-5 if basis == "f32" else 5e-2
    assert np.linalg.norm(np.eye(c.k) - V.T @ V) <= bound
    r = og.gmres_ir(A, b, 30, 1e-10, basis=basis, orth="dcgs2")
    ref = og.gmres_ir(A, b, 30, 1e-10, basis=basis)
    assert r.converged and r.rel_res <= 1e-10
    assert abs(r.iters - ref.iters) <= 30


def test_dcgs2_fp32_arnoldi_relation_under_cancellation():
    """Six tight eigenvalue clusters make the Krylov vectors nearly dependent, so in FP32 the first
    projection leaves a large component that the delayed pass must remove and the provisional
    Hessenberg columns must be corrected by -Hbar s (the t term).  The Arnoldi relation must still
    hold to a backward-stable FP32 level, 10 u sqrt(k) relative to ||H|| (a wrong sign of that
    correction gives ~1e-5 here; the correct code ~7e-8)."""
    rng = np.random.default_rng(0)
    d = np.concatenate([c + 1e-4 * rng.standard_normal(40) for c in [1, 2, 3, 5, 8, 13]])
    A = _diag_csr(d)
    r0 = rng.uniform(-1, 1, A.n)
    c = og.gmres_cycle_dcgs2(lambda z: og.spmv(A, z, np.float32), r0.astype(np.float32), 40,
                             dtype=np.float32)
    k = c.k
    V = c.V[:, : k + 1].astype(np.float64)
    AV = np.column_stack([og.spmv(A, V[:, i]) for i in range(k)])
    u32 = np.finfo(np.float32).eps / 2
    assert np.linalg.norm(AV - V @ c.H) <= 10 * u32 * np.sqrt(k) * np.linalg.norm(c.H)
    assert np.linalg.norm(np.eye(k + 1) - V.T @ V) <= 1e-5



def test_dcgs2_breakdown_norm_matches_a_v_under_cancellation():
    """The lucky-breakdown test of DCGS2 uses ||A v_j|| estimated as sqrt(||provisional column||^2
    + nu^2), the provisional column being (c - Hbar s) / nu with c's last entry (beta - s^T z) / nu.
    Under the strong cancellation of six tight eigenvalue clusters in FP32 the candidate's
    projections s are not small, and the estimate must match the directly computed ||A v_j||
    to 5 u (without the s^T z term it is off by ~2.6e-6 here; with it ~1.3e-7).  The final H
    does not separate the term: the next step's delayed pass absorbs it to first order."""
    rng = np.random.default_rng(0)
    d = np.concatenate([c + 1e-4 * rng.standard_normal(40) for c in [1, 2, 3, 5, 8, 13]])
    A = _diag_csr(d)
    r0 = rng.uniform(-1, 1, A.n)
    c = og.gmres_cycle_dcgs2(lambda z: og.spmv(A, z, np.float32), r0.astype(np.float32), 40,
                             dtype=np.float32)
    V = c.V.astype(np.float64)
    true = np.array([np.linalg.norm(og.spmv(A, V[:, i])) for i in range(c.k)])
    est = np.array(c.Az_norms[: c.k])
    u32 = np.finfo(np.float32).eps / 2
    assert np.max(np.abs(est - true) / true) <= 5 * u32
