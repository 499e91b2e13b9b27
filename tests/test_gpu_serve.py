"""Serving (mcs_submit / mcs_poll): continuous batching on one GPU.

Requests submitted while others run join them on the device; every request's
result must be the same alone and in the mix (sizes are exact integers, so
equal), each mapping must be valid, and a sample must match the CPU oracle."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[32, 8], ids=["warp-searchers", "8-lane-searchers"])
def solver(request):
    """One context per serving searcher width (the server launch takes it at
    the first submit)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06418_b300 import Solver
    s = Solver(0)
    s.set_serve_group(request.param)
    yield s
    s.close()


def _requests(count, seed=55, nmax=36):
    reqs = []
    for r in synth.config5_requests(count=count, rate_per_s=1e9, nmax=nmax, cid=seed):
        reqs.append(r.pair)
    return reqs


def _wait(solver, tickets, limit_s=120):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = solver.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < limit_s, "serving did not finish"
    return [out[t] for t in tickets]


def test_alone_equals_mix(solver):
    pairs = _requests(240)
    # alone: one request in flight at a time
    alone = []
    for p in pairs:
        t = solver.submit(p.G.adj, p.H.adj, p.G.labels, p.H.labels, timeout_s=20)
        alone += _wait(solver, [t])
    # mixed: submitted in waves while earlier ones run
    tickets = []
    for i in range(0, len(pairs), 40):
        for p in pairs[i:i + 40]:
            tickets.append(solver.submit(p.G.adj, p.H.adj, p.G.labels, p.H.labels, timeout_s=20))
        time.sleep(0.002)
    mixed = _wait(solver, tickets)
    for p, a, b in zip(pairs, alone, mixed):
        assert a.status == b.status == 0
        assert a.size == b.size
        assert oracle.verify(p.G.adj, p.H.adj, b.g_idx, b.h_idx, p.G.labels, p.H.labels) == 1
    for p, b in list(zip(pairs, mixed))[::6]:
        assert b.size == oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels).size


def _c5_golden():
    import itertools
    import json
    import os
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "golden", "c5_oracle.jsonl")
    if not os.path.exists(path):
        pytest.skip("c5_oracle.jsonl not generated")
    rows = [json.loads(x) for x in open(path)]
    sys.path.insert(0, os.path.join(here, "golden"))
    from make_oracle_golden import pair_digest
    n = max(r["idx"] for r in rows) + 1
    pairs = [r.pair for r in itertools.islice(synth.config5_requests(count=n), n)]
    for r in rows:
        assert r["digest"] == pair_digest(pairs[r["idx"]])
    return rows, pairs


def test_served_stream_matches_the_oracle_over_the_whole_size_range(solver):
    """The requests among the first 800 of the serving stream itself (n
    log-uniform in 16..56, 0-8 label classes) that the oracle proved within
    60 s -- 710, 375 of them with more than 36 vertices -- served together in
    waves with the oracle's own 60 s budget per request: each is proven by
    the server with the same size and a verified mapping.  (The 90 requests
    the oracle could not prove would hold searchers for the whole limit and
    say nothing exact.)  The proven requests of 37 or more vertices are then
    served again one at a time: alone equals in the mix."""
    from paper_1908_06418_b300 import MCS_OK
    rows, pairs = _c5_golden()
    rows = [r for r in rows if r["complete"]]
    tickets = []
    for i in range(0, len(rows), 100):
        for r in rows[i:i + 100]:
            p = pairs[r["idx"]]
            tickets.append(solver.submit(p.G.adj, p.H.adj, p.G.labels, p.H.labels, timeout_s=60))
        time.sleep(0.005)
    served = _wait(solver, tickets, limit_s=900)
    big = 0
    for r, res in zip(rows, served):
        p = pairs[r["idx"]]
        assert res.status == MCS_OK, (r["idx"], res.status)
        assert res.size == r["size"], (r["idx"], res.size, r["size"])
        assert oracle.verify(p.G.adj, p.H.adj, res.g_idx, res.h_idx, p.G.labels, p.H.labels) == 1
        big += int(max(p.G.n, p.H.n) > 36)
    assert big >= 300, big
    alone_rows = [(r, res) for r, res in zip(rows, served)
                  if max(pairs[r["idx"]].G.n, pairs[r["idx"]].H.n) > 36][:40]
    for r, res in alone_rows:
        p = pairs[r["idx"]]
        t = solver.submit(p.G.adj, p.H.adj, p.G.labels, p.H.labels, timeout_s=60)
        a = _wait(solver, [t])[0]
        assert a.status == MCS_OK and a.size == res.size == r["size"]


def test_serving_matches_batch_solver(solver):
    pairs = _requests(150, seed=56)
    batch = solver.solve_batch(pairs, timeout_s=20)
    tickets = [solver.submit(p.G.adj, p.H.adj, p.G.labels, p.H.labels, timeout_s=20) for p in pairs]
    served = _wait(solver, tickets)
    assert [r.size for r in served] == [r.size for r in batch]


def test_more_requests_than_slots_and_bad_input(solver):
    from paper_1908_06418_b300 import MCS_ERR_ARG
    pairs = _requests(2600, seed=57, nmax=20)            # > 2048 device slots
    bad = pairs[0].G.adj.copy()
    bad[0, 1] = 3
    tickets = [solver.submit(p.G.adj, p.H.adj, p.G.labels, p.H.labels, timeout_s=20) for p in pairs]
    tb = solver.submit(bad, pairs[0].H.adj, timeout_s=5)
    res = _wait(solver, tickets + [tb], limit_s=300)
    assert all(r.status == 0 for r in res[:-1])
    assert res[-1].status == MCS_ERR_ARG
    for p, r in list(zip(pairs, res))[::97]:
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1
    with pytest.raises(KeyError):
        solver.poll(tickets[0])                            # already released


def test_timeout_in_serving(solver):
    from paper_1908_06418_b300 import MCS_TIMEOUT
    p = synth.config4_pairs(count=1)[0]
    t = solver.submit(p.G.adj, p.H.adj, timeout_s=0.05)
    r = _wait(solver, [t])[0]
    assert r.status == MCS_TIMEOUT and r.size > 0
    assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx) == 1


def test_serve_group_is_fixed_once_serving(solver):
    p = _requests(1, seed=58)[0]
    t = solver.submit(p.G.adj, p.H.adj, p.G.labels, p.H.labels, timeout_s=20)
    _wait(solver, [t])
    with pytest.raises(ValueError):
        solver.set_serve_group(16)
    with pytest.raises(ValueError):
        solver.set_serve_group(4)

