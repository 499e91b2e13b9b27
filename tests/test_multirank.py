"""The multi-rank bench path on CPU: two gloo ranks, one shard of pairs each
(the search shards by pair with no exchange step, so ranks only agree on the
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


def _shard_rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import bench
    from make_oracle_golden import pair_digest
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        for name in ("c2", "td"):
            pairs, _ = bench.workload(name, shard=rank)
            out[name] = [(pair_digest(p), p.G.n, p.H.n, p.directed) for p in pairs]
        got = [None] * world
        dist.all_gather_object(got, out)
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_ranks_solve_disjoint_shards_of_the_same_recipe():
    """Under torchrun each rank solves its own shard: the workload's recipe
    (pair count, sizes, directedness) from seeds of its own, so the ranks
    share no pair; shard 0 is the workload the stored oracle optima cover."""
    import json
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res[0] == res[1]                      # every rank saw the same gathered shards
    shards = res[0]
    for name in ("c2", "td"):
        a, b = shards[0][name], shards[1][name]
        assert len(a) == len(b) > 0
        assert not {x[0] for x in a} & {x[0] for x in b}
        if name == "c2":                         # G(36, p) pairs: the same sizes per position
            assert [x[1:] for x in a] == [x[1:] for x in b]
        else:                                    # sizes drawn per pair: same directedness
            assert [x[3] for x in a] == [x[3] for x in b]
    rows = [json.loads(x) for x in open(os.path.join(ROOT, "tests", "golden", "c2_oracle.jsonl"))]
    assert [r["digest"] for r in sorted(rows, key=lambda r: r["idx"])] == [x[0] for x in shards[0]["c2"]]
