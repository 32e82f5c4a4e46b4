"""Block Jacobi with RCM ordering (Section III-D, Section V-G) against the oracle."""
import numpy as np
import pytest
import torch

import paper_2105_07544_b300 as g
import synth
from oracle import bjacobi as obj
from oracle import gmres as og
from gpu_util import dev, need_gpu

pytestmark = pytest.mark.gpu


def _problems():
    return [synth.permute_symmetric(synth.aniso2d(40, 0.02), 3),
            synth.convdiff2d(47, 0.9, peclet=60.0)]


@pytest.mark.parametrize("which", [0, 1])
def test_rcm_order_is_bit_exact(which):
    need_gpu()
    A = _problems()[which]
    s = g.Solver(A, m=20)
    s.set_block_jacobi(42)
    np.testing.assert_array_equal(s.block_jacobi_perm(), obj.rcm(A))
    s.close()


@pytest.mark.parametrize("k", [1, 7, 42, 64])
def test_apply_matches_the_oracle(k):
    need_gpu()
    A = _problems()[0]
    bj = obj.BlockJacobi(A, k)
    s = g.Solver(A, m=20)
    s.set_block_jacobi(k)
    v = synth.uniform(A.n, 11)
    z64 = s.precond_apply(dev(v), "f64").cpu().numpy()
    np.testing.assert_allclose(z64, bj.apply(v), rtol=1e-12, atol=1e-14 * np.abs(z64).max())
    z32 = s.precond_apply(dev(v).float(), "f32").cpu().numpy()
    ref32 = bj.apply(v, np.float32)
    assert np.abs(z32 - ref32).max() <= 1e-5 * np.abs(ref32).max()
    s.close()


@pytest.mark.parametrize("which", [0, 1])
def test_gmres_ir_with_block_jacobi_against_oracle(which):
    need_gpu()
    A = _problems()[which]
    b = synth.uniform(A.n, 5)
    ref = og.gmres_ir(A, b, 30, 1e-10, poly=obj.BlockJacobi(A, 42))
    assert ref.converged
    s = g.Solver(A, m=30)
    s.set_block_jacobi(42)
    x, st = s.ir_solve(dev(b), tol=1e-10)
    assert st.converged and abs(st.cycles - ref.cycles) <= 1
    assert np.linalg.norm(b - og.spmv(A, x.cpu().numpy())) / np.linalg.norm(b) <= 1e-10
    # fewer iterations than without the preconditioner
    s.set_block_jacobi(0)
    _, st0 = s.ir_solve(dev(b), tol=1e-10)
    assert st0.converged and st.iters < st0.iters
    s.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fp64_gmres_with_block_jacobi_against_oracle(prec):
    need_gpu()
    A = _problems()[0]
    b = synth.uniform(A.n, 8)
    ref = og.gmres(A, b, 30, 1e-10, poly=obj.BlockJacobi(A, 42),
                   poly_dtype=np.float32 if prec == "f32" else None)
    assert ref.converged
    s = g.Solver(A, m=30, fp64_precond=prec)
    s.set_block_jacobi(42)
    x, st = s.solve_fp64(dev(b), tol=1e-10)
    s.close()
    assert st.converged and st.rel_res <= 1e-10
    assert abs(st.iters - ref.iters) <= 30
    assert np.linalg.norm(b - og.spmv(A, x.cpu().numpy())) / np.linalg.norm(b) <= 1e-10


def test_invalid_block_jacobi_requests():
    need_gpu()
    A = synth.laplace2d(20)
    s = g.Solver(A, m=10)
    with pytest.raises(g.GmresError):
        s.set_block_jacobi(65)
    s.close()
    sp = g.Solver(A, m=10, poly_degree=5, poly_start=synth.poly_start_vector(A.n))
    with pytest.raises(g.GmresError):
        sp.set_block_jacobi(4)
    sp.close()
    # a matrix with a zero diagonal entry has a singular 1 x 1 block
    Z = synth._from_coo(3, [0, 0, 1, 1, 2], [0, 1, 0, 2, 2], [0.0, 1.0, 1.0, 1.0, 2.0], "z")
    sz = g.Solver(Z, m=2)
    with pytest.raises(g.GmresError):
        sz.set_block_jacobi(1)
    sz.close()
