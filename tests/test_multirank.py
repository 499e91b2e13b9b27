"""The multi-rank bench path on CPU: two gloo ranks, one replica each (the
search shards by pair with no exchange step, so ranks only agree on the
timing and the summed work).  No GPU needed."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed (r + 1) * 100 ms for 10 + r solved pairs and 1000 * (r + 1) nodes
        out = bench.combine_ranks(100.0 * (rank + 1), 10 + rank, 1000 * (rank + 1), dist, "cpu")
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_slowest_time_and_summed_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    for r in (0, 1):
        assert res[r] == (200.0, 21, 3000)


def test_one_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(12.5, 3, 44) == (12.5, 3, 44)
