"""Pins of the block Jacobi / RCM oracle (CPU)."""
import numpy as np
import pytest

import synth
from oracle import bjacobi as obj
from oracle import gmres as og


def _graph(n, edges):
    rows = [i for i in range(n)] + [a for a, b in edges] + [b for a, b in edges]
    cols = [i for i in range(n)] + [b for a, b in edges] + [a for a, b in edges]
    vals = [4.0] * n + [-1.0] * (2 * len(edges))
    return synth._from_coo(n, rows, cols, vals, "graph")


def test_rcm_hand_checked_small_graph():
    # degrees 0:2 1:2 2:2 3:3 4:1; start at 4 (smallest degree); BFS 4 -> 3 -> (1, 2) -> 0;
    # Cuthill-McKee order [4, 3, 1, 2, 0], reversed
    A = _graph(5, [(0, 1), (0, 2), (1, 3), (2, 3), (3, 4)])
    np.testing.assert_array_equal(obj.rcm(A), [0, 2, 1, 3, 4])


def test_rcm_recovers_a_shuffled_path_and_is_a_permutation():
    n = 200
    rng = np.random.default_rng(1)
    lab = rng.permutation(n)
    A = _graph(n, [(int(lab[i]), int(lab[i + 1])) for i in range(n - 1)])
    p = obj.rcm(A)
    np.testing.assert_array_equal(np.sort(p), np.arange(n))
    assert obj.bandwidth(A) > 50 and obj.bandwidth(A, p) == 1


def test_rcm_bandwidth_of_a_shuffled_grid_is_near_the_natural_one():
    N = 30
    A = synth.permute_symmetric(synth.laplace2d(N), 3)
    p = obj.rcm(A)
    assert obj.bandwidth(A) > 10 * N
    assert obj.bandwidth(A, p) <= 2 * N
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    M = sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.n, A.n))
    q = reverse_cuthill_mckee(M, symmetric_mode=True)
    assert obj.bandwidth(A, p) <= 1.5 * obj.bandwidth(A, q)


def test_rcm_handles_disconnected_components():
    A = _graph(6, [(0, 1), (3, 4), (4, 5)])          # components {0,1}, {2}, {3,4,5}
    p = obj.rcm(A)
    np.testing.assert_array_equal(np.sort(p), np.arange(6))
    assert obj.bandwidth(A, p) <= 1


def test_block_size_one_is_diagonal_scaling_and_full_block_is_the_inverse():
    A = synth.convdiff2d(12, 0.3, peclet=50.0)
    v = synth.uniform(A.n, 4)
    diag = np.array([A.val[A.rowptr[i]:A.rowptr[i + 1]][A.colidx[A.rowptr[i]:A.rowptr[i + 1]] == i][0]
                     for i in range(A.n)])
    np.testing.assert_allclose(obj.BlockJacobi(A, 1).apply(v), v / diag, rtol=1e-15)
    full = obj.BlockJacobi(A, A.n)
    import scipy.sparse as sp
    M = sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.n, A.n)).toarray()
    np.testing.assert_allclose(full.apply(v), np.linalg.solve(M, v), rtol=1e-10, atol=1e-12)
    # right preconditioning with the exact inverse: GMRES finishes in one step
    r = og.gmres(A, v, 10, 1e-10, poly=full)
    assert r.converged and r.iters == 1


def test_block_jacobi_equals_block_diagonal_of_the_permuted_matrix():
    A = synth.permute_symmetric(synth.aniso2d(16, 0.05), 2)
    k = 42
    bj = obj.BlockJacobi(A, k)
    import scipy.sparse as sp
    M = sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.n, A.n)).toarray()
    P = M[bj.perm][:, bj.perm]                         # P A P^T
    D = np.zeros_like(P)
    for b0 in range(0, A.n, k):
        D[b0:b0 + k, b0:b0 + k] = P[b0:b0 + k, b0:b0 + k]
    v = synth.uniform(A.n, 6)
    z = np.empty(A.n)
    z[bj.perm] = np.linalg.solve(D, v[bj.perm])
    np.testing.assert_allclose(bj.apply(v), z, rtol=1e-12, atol=1e-14)


def test_block_jacobi_speeds_up_gmres_ir_on_a_shuffled_anisotropic_problem():
    A = synth.permute_symmetric(synth.aniso2d(32, 0.01), 5)
    b = synth.uniform(A.n, 7)
    r0 = og.gmres_ir(A, b, 30, 1e-10)
    r42 = og.gmres_ir(A, b, 30, 1e-10, poly=obj.BlockJacobi(A, 42))
    assert r0.converged and r42.converged and r42.rel_res <= 1e-10
    assert r42.iters < r0.iters


def test_block_jacobi_on_heterogeneous_coefficients():
    """Row scales spread over 1e4: diagonal (k = 1) and block (k = 42) Jacobi cut the GMRES-IR
    iterations several-fold on the relabelled problem."""
    A = synth.permute_symmetric(synth.hetero2d(40, 1e4, 0), 1)
    b = synth.uniform(A.n, 7)
    r0 = og.gmres_ir(A, b, 30, 1e-10, maxiter=20000)
    for k in (1, 42):
        r = og.gmres_ir(A, b, 30, 1e-10, poly=obj.BlockJacobi(A, k))
        assert r.converged and r.rel_res <= 1e-10
        assert 5 * r.iters < r0.iters
