"""The N > 1 path of bench.py on the CPU: two gloo ranks (replicas / weak
scaling, no collective on the data path, max-over-ranks time, summed work)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        insts, desc = bench.make_workload("batch", rank, n_batch=8)
        first = [float(i.m0[0, :4].sum()) for i in insts]
        dt, upd = bench.reduce_over_ranks(1.0 + rank, 100 + 10 * rank, dist, "cpu")
        q.put((rank, dt, upd, first, desc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_batch_and_reduce_time_and_work():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    # every rank reports the slowest rank's time and the sum of the updates
    for _, dt, upd, _, _ in out:
        assert dt == 2.0 and upd == 210.0
    # each rank advances its own seeded batch (no shared instances)
    assert out[0][3] != out[1][3]
