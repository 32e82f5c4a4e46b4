"""The benchmark's multi-rank logic with world_size 2 over gloo on CPU: rendezvous on 127.0.0.1,
barrier, max-over-ranks timing, and per-rank workloads (independent replicas / shards, no
collective on the data path)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    import synth
    w, r = bench.dist_setup()
    bench.barrier(w)
    t = bench.max_over_ranks(1.0 + r, w)                 # slowest rank's time
    b = synth.uniform(64, r)                              # the bench seeds each rank's b by rank
    sys_r = synth.workload_batched(nsys=2, side_lo=4, side_hi=6, seed0=1000 * r)   # and its batch
    out.put((r, w, t, float(b[0]), float(sys_r[0][1][0, 0])))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=240) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2, 2]
    assert res[0][2] == res[1][2] == 2.0                  # max over ranks
    assert res[0][3] != res[1][3] and res[0][4] != res[1][4]   # each rank its own inputs
