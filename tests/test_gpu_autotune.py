"""Launch-shape autotuner: every candidate shape solves to the FP64 tolerance with the oracle's
iteration count (to within one cycle: the shapes regroup FP32 partial sums), the tuner keeps a
shape no slower than the default, and the cache reapplies it."""
import numpy as np
import pytest
import torch

import paper_2105_07544_b300 as g
import synth
from oracle import gmres as og
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

M = 30


@pytest.fixture(scope="module")
def problem():
    A = synth.laplace3d(48)                     # n = 110,592: 864 tiles, many groups per CTA
    b = synth.uniform(A.n, 7)
    ref = og.gmres_ir(A, b, M, 1e-10)
    assert ref.converged
    return A, b, ref


SHAPES = [dict(sweep_stage_kb=a, sweep_ctas_per_sm=c, spmv_ctas_per_sm=s)
          for a in (0, 8, 32) for c in (0, 1, 3) for s in (0, 4)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda d: "-".join(str(v) for v in d.values()))
def test_every_shape_reaches_the_oracle(problem, shape):
    need_gpu()
    A, b, ref = problem
    s = g.Solver(A, m=M)
    s.set_tuning(**shape)
    assert {k: s.get_tuning()[k] for k in shape} == shape
    x, st = s.ir_solve(torch.from_numpy(b).cuda(), tol=1e-10)
    s.close()
    assert st.converged and st.rel_res <= 1e-10
    assert abs(st.iters - ref.iters) <= M


def test_autotune_keeps_a_shape_no_slower_than_default(problem, tmp_path):
    need_gpu()
    from paper_2105_07544_b300 import autotune as at
    A, b, ref = problem
    bd = torch.from_numpy(b).cuda()
    s = g.Solver(A, m=M)
    cache = at.TuningCache(str(tmp_path / "t.json"))
    r = at.tune(s, bd, A.nnz, "f32", 0, cache)
    assert not r["cached"] and r["s_per_iter"] <= r["default_s_per_iter"]
    assert s.get_tuning() == r["shapes"]
    x, st = s.ir_solve(bd, tol=1e-10)
    assert st.converged and abs(st.iters - ref.iters) <= M
    s.close()
    s2 = g.Solver(A, m=M)
    r2 = at.tune(s2, bd, A.nnz, "f32", 0, at.TuningCache(str(tmp_path / "t.json")))
    assert r2["cached"] and s2.get_tuning() == r["shapes"]
    s2.close()


def test_invalid_shapes_are_rejected():
    need_gpu()
    s = g.Solver(synth.laplace2d(16), m=10)
    for bad in (dict(sweep_ctas_per_sm=5), dict(spmv_ctas_per_sm=-1), dict(sweep_stage_kb=1000),
                dict(spmv_lanes_per_row=6)):
        with pytest.raises(g.GmresError):
            s.set_tuning(**bad)
    s.close()
