"""The N > 1 path of the benchmark on CPU: two gloo ranks, each with its own
batch, reduce to the slowest rank's time and the sum of clusters (no
collective touches the tracking data)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, n = bench.aggregate_ranks(100.0 + 25.0 * rank, 1000 + rank, world)
    q.put((rank, ms, n))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, n in res:
        assert ms == 125.0 and n == 2001


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_ranks(7.5, 42, 1) == (7.5, 42)
