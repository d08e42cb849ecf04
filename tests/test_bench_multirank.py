"""The multi-rank path of bench.py on CPU: two gloo ranks, weak scaling, max over ranks."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.aggregate_max(0.5 + rank)          # rank 1 is slower
    rate = bench.whole_job_rate(1000, world, 10, t)
    wl = bench.workload(rank, frames=1)
    out.put((rank, t, rate, wl.total, int(wl.data[:64].astype("int64").sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=300) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, n0, s0), (r1, t1, v1, n1, s1) = res
    assert t0 == t1 == 1.5                      # max over ranks
    assert v0 == v1 == 1000 * 2 * 10 / 1.5      # whole-job units over the slowest rank
    assert n0 == n1                              # same shape on every rank (weak scaling) ...
    assert s0 != s1                              # ... from different seeds


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate_max(2.25) == 2.25
    assert bench.whole_job_rate(10, 1, 3, 2.0) == 15.0
