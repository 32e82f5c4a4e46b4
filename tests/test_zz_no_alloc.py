"""The allocation-free polynomial entry point (needs a GPU).

gmres_precond_apply_noalloc serves callers that may not allocate device memory while they run
(a memory pool or arena that owns the GPU, a real-time loop that cannot afford cudaMalloc's
implicit synchronisation, a plug-in whose host forbids allocation).  It must give the same
z = p(A) v as the allocating gmres_precond_apply, on consecutive calls that reuse its fixed
scratch array, and must refuse problems larger than that array.  This file sorts last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2105_07544_b300 as g
import synth
from gpu_util import dev, need_gpu

pytestmark = pytest.mark.gpu


def _noalloc(lib, solver, prec, v):
    z = torch.empty_like(v)
    torch.cuda.synchronize()
    rc = lib.gmres_precond_apply_noalloc(solver.h, g._PREC[prec], ctypes.c_void_p(v.data_ptr()),
                                         ctypes.c_void_p(z.data_ptr()))
    torch.cuda.synchronize()
    return rc, z


@pytest.mark.parametrize("prec,dtype", [("f64", torch.float64), ("f32", torch.float32)])
def test_noalloc_matches_allocating_entry_point_twice(prec, dtype):
    """Both entry points run the same polynomial steps on the same matrix copy with the same
    coefficients, each row computed by itself: the results agree bit for bit, on two calls in a
    row (the second finds the first call's vectors still in the scratch array)."""
    need_gpu()
    lib = g.load()
    A = synth.convdiff2d(97, 1.3, 100.0)                   # n = 9409, ragged last tile
    start = synth.poly_start_vector(A.n, 0)
    s = g.Solver(A, m=30, poly_degree=10, poly_start=start)
    for call in range(2):                                   # the scratch keeps the last call's data
        v = dev(synth.uniform(A.n, 40 + call), dtype)
        ref = s.precond_apply(v, prec)
        torch.cuda.synchronize()
        rc, z = _noalloc(lib, s, prec, v)
        assert rc == 0, g.status_string(rc)
        assert torch.isfinite(z).all()
        assert torch.equal(z, ref)
    s.close()


def test_noalloc_refuses_an_output_that_overlaps_its_input():
    need_gpu()
    lib = g.load()
    A = synth.convdiff2d(40, 0.3, 100.0)
    s = g.Solver(A, m=10, poly_degree=4, poly_start=synth.poly_start_vector(A.n, 0))
    v = dev(synth.uniform(2 * A.n, 5))
    torch.cuda.synchronize()
    for off in (0, 7, A.n - 1):                             # z == v and partial overlaps
        rc = lib.gmres_precond_apply_noalloc(s.h, g._PREC["f64"], ctypes.c_void_p(v.data_ptr()),
                                             ctypes.c_void_p(v.data_ptr() + 8 * off))
        assert rc == -1                                     # GMRES_ERR_INVALID_ARG
    rc = lib.gmres_precond_apply_noalloc(s.h, g._PREC["f64"], ctypes.c_void_p(v.data_ptr()),
                                         ctypes.c_void_p(v.data_ptr() + 8 * A.n))
    torch.cuda.synchronize()
    assert rc == 0                                          # adjacent, not overlapping
    s.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    need_gpu()
    lib = g.load()
    A = synth.laplace2d(800)                                # n = 640,000 > 524,288
    s = g.Solver(A, m=4, poly_degree=2, poly_start=synth.poly_start_vector(A.n, 0))
    v = dev(np.ones(A.n))
    rc, _ = _noalloc(lib, s, "f64", v)
    assert rc == -1                                         # GMRES_ERR_INVALID_ARG
    s.close()
