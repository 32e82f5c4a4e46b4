"""Batched block GMRES-IR against the oracle (needs a GPU): many uneven convection-diffusion
systems with 8 right-hand sides each, solved together."""
import numpy as np
import pytest
import torch

import paper_2105_07544_b300 as g
import synth
from oracle import block as ob
from oracle import gmres as og
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_batch():
    return synth.workload_batched(nsys=12, side_lo=12, side_hi=45, seed0=100)


def test_batch_small_against_oracle(small_batch):
    need_gpu()
    systems = [A for A, _ in small_batch]
    Bs = [B for _, B in small_batch]
    bs = g.BatchSolver(systems, m=8)
    x, st = bs.ir_solve(bs.pack(Bs), tol=1e-10)
    assert st.converged and st.converged_systems == len(systems)
    assert st.max_rel_res <= 1e-10
    Xs = bs.unpack(x)
    for (A, B), X in zip(small_batch, Xs):
        R = B - ob.spmm(A, X)
        rel = np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)
        assert np.all(rel <= 1e-10)
        Xo = np.column_stack([og.gmres(A, B[:, c], 60, 1e-13).x for c in range(8)])
        assert np.linalg.norm(X - Xo) <= 1e-7 * np.linalg.norm(Xo)
    # block-IR cycle counts of the oracle (same restart length) as a sanity range
    A0, B0 = small_batch[0]
    ro = ob.block_gmres_ir(A0, B0, 8, 1e-10, basis="bf16")
    assert st.per_system_cycles[0] <= 2 * ro.cycles + 2
    bs.close()


def test_batch_device_buffers_and_resume(small_batch):
    need_gpu()
    systems = [A for A, _ in small_batch]
    bs = g.BatchSolver(systems, m=8)
    Bflat = torch.from_numpy(bs.pack([B for _, B in small_batch])).cuda()
    x1, s1 = bs.ir_solve(Bflat, tol=1e-10)
    assert s1.converged
    xh, sh = bs.ir_solve(Bflat.cpu().numpy(), tol=1e-10)
    assert np.array_equal(x1.cpu().numpy(), xh)           # deterministic
    x2, s2 = bs.ir_solve(Bflat, X=x1.clone(), tol=1e-10)  # resume from a converged iterate
    assert s2.converged and s2.cycles == 0
    bs.close()


def test_batch_profiling_mode_matches_graphs_bitwise(small_batch):
    """Direct launches with event timing run the same kernels in the same order as the graph:
    identical iterates; every kernel class is timed."""
    need_gpu()
    systems = [A for A, _ in small_batch]
    bs = g.BatchSolver(systems, m=8)
    Bflat = torch.from_numpy(bs.pack([B for _, B in small_batch])).cuda()
    x1, s1 = bs.ir_solve(Bflat, tol=1e-10)
    bs.set_profiling(True)
    x2, s2 = bs.ir_solve(Bflat, tol=1e-10)
    bs.set_profiling(False)
    assert s1.converged and s2.converged and s1.cycles == s2.cycles
    assert torch.equal(x1, x2)
    assert all(v > 0 for v in s2.t_kernel.values())
    assert s2.class_launches["sweep"] == 3 * 8 * s2.cycles
    assert s2.class_launches["spmm"] == 8 * s2.cycles
    bs.close()


def test_batched_bench_workload_sizes_in_bounds():
    """The benchmark's batched workload is 256 systems of sides 32..320 (checked on the host)."""
    wl = synth.workload_batched()
    assert len(wl) == 256
    sides = [int(round(np.sqrt(A.n))) for A, _ in wl]
    assert min(sides) >= 32 and max(sides) <= 320


@pytest.fixture(scope="module")
def tiled_batch():
    """Systems of 31-79 tiles, so that every chunk size splits them into several chunks with a
    ragged last chunk; the oracle's FP64 GMRES solution of the largest one."""
    wl = synth.workload_batched(nsys=6, side_lo=60, side_hi=110, seed0=300)
    big = max(range(len(wl)), key=lambda i: wl[i][0].n)
    A, B = wl[big]
    Xo = np.column_stack([og.gmres(A, B[:, c], 60, 1e-13).x for c in range(8)])
    return wl, big, Xo


BATCH_SHAPES = [dict(chunk_tiles=c, sweep_smem_kb=k, sweep_max_stages=st)
                for c, k, st in ((0, 0, 0), (4, 64, 2), (8, 0, 8), (32, 220, 8), (64, 160, 3))]


def _check_batch_solution(wl, Xs, tol):
    for (A, B), X in zip(wl, Xs):
        R = B - ob.spmm(A, X)
        rel = np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)
        assert np.all(rel <= tol)


@pytest.mark.parametrize("shape", BATCH_SHAPES, ids=lambda d: "-".join(str(v) for v in d.values()))
def test_batch_launch_shapes_reach_the_oracle(tiled_batch, shape):
    """Every launch shape solves every column to the FP64 tolerance (residuals by the oracle's
    FP64 SpMM) and agrees with the oracle's solution of the largest system."""
    need_gpu()
    wl, big, Xo = tiled_batch
    bs = g.BatchSolver([A for A, _ in wl], m=8)
    bs.set_tuning(**shape)
    assert bs.get_tuning() == shape
    x, st = bs.ir_solve(bs.pack([B for _, B in wl]), tol=1e-10)
    assert st.converged and st.converged_systems == len(wl) and st.max_rel_res <= 1e-10
    Xs = bs.unpack(x)
    _check_batch_solution(wl, Xs, 1e-10)
    assert np.linalg.norm(Xs[big] - Xo) <= 1e-7 * np.linalg.norm(Xo)
    bs.close()


def test_batch_shape_changes_between_solves(tiled_batch):
    """Changing the chunk size on a live batch (reallocated partial sums, new graph) and changing
    it back reproduces the first solve bit for bit."""
    need_gpu()
    wl, _, _ = tiled_batch
    bs = g.BatchSolver([A for A, _ in wl], m=8)
    Bf = bs.pack([B for _, B in wl])
    x1, s1 = bs.ir_solve(Bf, tol=1e-10)
    bs.set_tuning(chunk_tiles=4)
    x2, s2 = bs.ir_solve(Bf, tol=1e-10)
    bs.set_tuning(chunk_tiles=0)
    x3, s3 = bs.ir_solve(Bf, tol=1e-10)
    assert s1.converged and s2.converged and s3.converged
    assert np.array_equal(x1, x3) and s1.cycles == s3.cycles
    _check_batch_solution(wl, bs.unpack(x2), 1e-10)
    bs.close()


def test_batch_autotune_keeps_a_shape_no_slower_than_default(tiled_batch, tmp_path):
    need_gpu()
    from paper_2105_07544_b300 import autotune as at
    wl, _, _ = tiled_batch
    bs = g.BatchSolver([A for A, _ in wl], m=8)
    Bd = torch.from_numpy(bs.pack([B for _, B in wl])).cuda()
    nnz = sum(int(A.nnz) for A, _ in wl)
    r = at.tune_batch(bs, Bd, nnz, 8, cache=at.TuningCache(str(tmp_path / "t.json")))
    assert not r["cached"] and r["s_per_iter"] <= r["default_s_per_iter"]
    assert bs.get_tuning() == r["shapes"]
    assert r["shapes"]["chunk_tiles"] in (0, 8, 32)
    x, st = bs.ir_solve(Bd, tol=1e-10)
    assert st.converged
    _check_batch_solution(wl, bs.unpack(x), 1e-10)
    bs.close()


def test_batch_invalid_shapes_are_rejected(small_batch):
    need_gpu()
    bs = g.BatchSolver([A for A, _ in small_batch], m=8)
    before = bs.get_tuning()
    for bad in (dict(chunk_tiles=3), dict(chunk_tiles=65), dict(sweep_smem_kb=63),
                dict(sweep_smem_kb=221), dict(sweep_max_stages=1), dict(sweep_max_stages=9)):
        with pytest.raises(g.GmresError):
            bs.set_tuning(**bad)
        assert bs.get_tuning() == before
    bs.close()


def test_batch_edge_cases_tiny_systems_zero_columns_and_converged_starts():
    """One-tile systems (n = 9 and 1), a zero right-hand-side column (its solution stays zero),
    and a system started from its oracle solution (it converges at the first residual, while the
    others run) in one batch."""
    need_gpu()
    wl = synth.workload_batched(nsys=3, side_lo=20, side_hi=40, seed0=700)
    A1 = synth.convdiff2d(3, 0.3, 100.0, 0.2)                         # n = 9
    A0 = synth.CSR(n=1, rowptr=np.array([0, 1], np.int32), colidx=np.array([0], np.int32),
                   val=np.array([2.5]))
    rng = np.random.default_rng(701)
    B1 = rng.uniform(-1.0, 1.0, (A1.n, 8))
    B1[:, 3] = 0.0
    B0 = rng.uniform(-1.0, 1.0, (1, 8))
    systems = [A for A, _ in wl] + [A1, A0]
    Bs = [B for _, B in wl] + [B1, B0]
    # system 0 starts at its oracle solution
    X0 = [np.zeros_like(B) for B in Bs]
    X0[0] = np.column_stack([og.gmres(systems[0], Bs[0][:, c], 60, 1e-14).x for c in range(8)])
    bs = g.BatchSolver(systems, m=8)
    x, st = bs.ir_solve(bs.pack(Bs), X=bs.pack(X0), tol=1e-10)
    assert st.converged and st.converged_systems == len(systems)
    assert st.per_system_cycles[0] == 0 and max(st.per_system_cycles[1:]) >= 1
    Xs = bs.unpack(x)
    for A, B, X in zip(systems, Bs, Xs):
        R = B - ob.spmm(A, X)
        nb = np.linalg.norm(B, axis=0)
        assert np.all(np.linalg.norm(R, axis=0) <= 1e-10 * np.where(nb > 0, nb, 1.0))
    assert np.all(Xs[3][:, 3] == 0.0)
    assert np.allclose(Xs[4], B0 / 2.5, rtol=1e-9, atol=0)      # tol 1e-10 on a 1 x 1 system
    bs.close()
