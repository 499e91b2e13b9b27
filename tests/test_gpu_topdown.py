"""The top-down strategy (Section IV-A) on the GPU against the oracle: the
optimum must equal the plain search's, a lone searcher must walk the oracle's
goal searches node for node, and time limits must report verified mappings."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06418_b300 import Solver
    s = Solver(0)
    yield s
    s.close()


def _pairs(count, nmin, nmax, seed, directed=False, k=0, pmin=0.1, pmax=0.6):
    rs = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nG, nH = int(rs.integers(nmin, nmax + 1)), int(rs.integers(nmin, nmax + 1))
        p = float(rs.uniform(pmin, pmax))
        rg, rh = synth.rng_for(seed, i, 0), synth.rng_for(seed, i, 1)
        f = synth.er_directed if directed else synth.er_undirected
        out.append(synth.Pair(synth.Graph(f(nG, p, rg), synth.uniform_labels(nG, k, rg)),
                              synth.Graph(f(nH, p, rh), synth.uniform_labels(nH, k, rh)), directed))
    return out


@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 3)])
def test_topdown_batch_equals_oracle(solver, directed, k):
    from paper_1908_06418_b300 import MCS_TOP_DOWN
    pairs = _pairs(150, 2, 22, 3100 + k + (50 if directed else 0), directed, k)
    res = solver.solve_batch(pairs, flags=MCS_TOP_DOWN, directed=directed, timeout_s=60)
    for i, (p, r) in enumerate(zip(pairs, res)):
        o = oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed)
        assert r.status == 0, (i, r.status)
        assert r.size == o.size, (i, r.size, o.size)
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1, i


@pytest.mark.parametrize("group", [32, 8, 4])
@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 3)])
def test_topdown_single_searcher_walks_the_oracle_goal_searches(solver, group, directed, k):
    """One searcher, no per-sibling bound re-test: every goal search visits
    the oracle's nodes, the re-enqueued root included, and stops at the node
    that reaches the goal; the counts summed over the goals are equal."""
    from paper_1908_06418_b300 import MCS_TOP_DOWN, MCS_NO_LEVEL_PRUNE
    pairs = _pairs(30, 3, 16, 3300 + k + (50 if directed else 0), directed, k)
    solver.set_max_warps(1)
    solver.set_search_group(group)
    try:
        for i, p in enumerate(pairs):
            r = solver.solve(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed,
                             flags=MCS_TOP_DOWN | MCS_NO_LEVEL_PRUNE, timeout_s=30)
            o = oracle.mcs_topdown(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed)
            assert r.status == 0 and o.complete
            assert r.size == o.size, (i, r.size, o.size)
            assert r.nodes == o.nodes, (i, r.nodes, o.nodes)
            assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1
    finally:
        solver.set_max_warps(0)
        solver.set_search_group(8)


def test_topdown_maps_an_induced_subgraph_at_the_first_goal(solver):
    from paper_1908_06418_b300 import MCS_TOP_DOWN
    rs = np.random.default_rng(3500)
    pairs = []
    for i in range(40):
        n = int(rs.integers(10, 40))
        b = synth.er_undirected(n + 8, float(rs.uniform(0.1, 0.5)), synth.rng_for(3500, i, 0))
        keep = np.sort(rs.permutation(n + 8)[:n])
        pairs.append(synth.Pair(synth.Graph(b[np.ix_(keep, keep)].copy()), synth.Graph(b)))
    res = solver.solve_batch(pairs, flags=MCS_TOP_DOWN, timeout_s=60)
    for p, r in zip(pairs, res):
        assert r.status == 0 and r.size == p.G.n
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx) == 1


def test_topdown_time_limit_reports_a_verified_mapping(solver):
    from paper_1908_06418_b300 import MCS_TOP_DOWN, MCS_TIMEOUT
    pairs = synth.config4_pairs(count=8)
    res = solver.solve_batch(pairs, flags=MCS_TOP_DOWN, timeout_s=0.05)
    for p, r in zip(pairs, res):
        assert r.status in (0, MCS_TIMEOUT)
        assert len(r.g_idx) == r.size
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx) == 1


def test_topdown_mixed_with_edge_cases(solver):
    """Empty graphs, a single vertex, disjoint labels and malformed input in
    one top-down batch."""
    from paper_1908_06418_b300 import MCS_TOP_DOWN, MCS_ERR_ARG
    e = np.zeros((0, 0), np.uint8)
    one = np.zeros((1, 1), np.uint8)
    bad = np.full((3, 3), 2, np.uint8)
    a = synth.er_undirected(12, 0.4, synth.rng_for(3600, 0, 0))
    pairs = [(e, a, None, None), (one, one, None, None), (a, a, np.zeros(12, np.int32), np.ones(12, np.int32)),
             (bad, a, None, None), (a, a, None, None)]
    res = solver.solve_batch(pairs, flags=MCS_TOP_DOWN, timeout_s=10)
    assert [r.status for r in res] == [0, 0, 0, MCS_ERR_ARG, 0]
    assert [r.size for r in res] == [0, 1, 0, 0, 12]


def test_topdown_is_rejected_by_the_server(solver):
    from paper_1908_06418_b300 import MCS_TOP_DOWN
    a = synth.er_undirected(10, 0.3, synth.rng_for(3700, 0, 0))
    with pytest.raises(Exception):
        solver.submit(a, a, flags=MCS_TOP_DOWN)


# --------------------------------------------------------------------------
# dead-end forecasting with a bound increase and a binary search (Section IV-A)
# --------------------------------------------------------------------------
def _golden(name):
    import json
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "golden", name)) as f:
        return [json.loads(l) for l in f if l.strip()]


@pytest.mark.parametrize("threshold,doubling", [(64, 0), (1024, 0), (64, 1), (4096, 1)])
def test_deadend_labelled_batch_equals_stored_oracle(solver, threshold, doubling):
    """512 pairs of the labelled batch with thresholds low enough that pairs
    raise their bound (and some raise it past the optimum, which the binary
    search must then recover): every size equals the stored oracle optimum."""
    from paper_1908_06418_b300 import MCS_DEAD_END
    rows = {r["idx"]: r for r in _golden("c3_oracle.jsonl")}
    pairs = synth.config3_pairs()[:512]
    solver.set_dead_end(threshold, doubling)
    try:
        res = solver.solve_batch(pairs, flags=MCS_DEAD_END, timeout_s=60)
    finally:
        solver.set_dead_end(-1, -1)
    for i, (p, r) in enumerate(zip(pairs, res)):
        g = rows[i]
        assert r.status == 0, (i, r.status)
        assert r.size == g["size"] if g["complete"] else r.size >= g["size"], (i, r.size, g["size"])
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1, i


@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 3)])
def test_deadend_small_threshold_batch_equals_oracle(solver, directed, k):
    from paper_1908_06418_b300 import MCS_DEAD_END
    pairs = _pairs(120, 8, 24, 3800 + k + (50 if directed else 0), directed, k)
    solver.set_dead_end(32, 0)
    try:
        res = solver.solve_batch(pairs, flags=MCS_DEAD_END, directed=directed, timeout_s=60)
    finally:
        solver.set_dead_end(-1, -1)
    for i, (p, r) in enumerate(zip(pairs, res)):
        o = oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed)
        assert r.status == 0 and r.size == o.size, (i, r.size, o.size)
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1, i


def test_deadend_never_reached_is_the_plain_search(solver):
    """With a threshold no pair reaches, a lone searcher walks the plain
    search tree node for node."""
    from paper_1908_06418_b300 import MCS_DEAD_END, MCS_NO_LEVEL_PRUNE
    pairs = _pairs(20, 4, 16, 3900)
    solver.set_max_warps(1)
    solver.set_dead_end(1 << 50, 0)
    try:
        for p in pairs:
            r = solver.solve(p.G.adj, p.H.adj, flags=MCS_DEAD_END | MCS_NO_LEVEL_PRUNE, timeout_s=30)
            o = oracle.mcs(p.G.adj, p.H.adj)
            assert r.status == 0 and r.size == o.size and r.nodes == o.nodes
    finally:
        solver.set_max_warps(0)
        solver.set_dead_end(-1, -1)


def test_deadend_parameters_and_flag_combination(solver):
    import torch
    from paper_1908_06418_b300 import MCS_DEAD_END, MCS_TOP_DOWN, MCS_ERR_ARG, DeviceBatch
    for bad in ((0, 0), (-2, 0), (100, 2), (100, -2)):
        with pytest.raises(ValueError):
            solver.set_dead_end(*bad)
    pairs = _pairs(4, 6, 10, 3950)
    b = DeviceBatch(pairs)
    n = len(pairs)
    out = [torch.zeros(n, dtype=torch.int32, device=b.device), torch.zeros(n, dtype=torch.int32, device=b.device),
           torch.zeros(n, dtype=torch.int64, device=b.device)]
    rc = solver.solve_batch_device(n, b.d_n, b.d_adj_off, b.d_adj, b.d_lab_off, b.d_labels, *out,
                                   flags=b.flags | MCS_DEAD_END | MCS_TOP_DOWN, timeout_s=10)
    assert rc == MCS_ERR_ARG


# --------------------------------------------------------------------------
# randomized restarts (Section IV-A)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("min_nodes,seed", [(64, 0), (4096, 77)])
def test_restart_labelled_batch_equals_stored_oracle(solver, min_nodes, seed):
    """Restarts that fire after a few polls: every open branch of the
    restarting searcher goes back to the ring, and no part of the tree may
    be lost -- the sizes equal the stored oracle optima."""
    from paper_1908_06418_b300 import MCS_RESTART
    rows = {r["idx"]: r for r in _golden("c3_oracle.jsonl")}
    pairs = synth.config3_pairs()[:512]
    solver.set_restart(min_nodes, seed)
    try:
        res = solver.solve_batch(pairs, flags=MCS_RESTART, timeout_s=60)
    finally:
        solver.set_restart(-1, 0)
    for i, (p, r) in enumerate(zip(pairs, res)):
        g = rows[i]
        assert r.status == 0, (i, r.status)
        assert r.size == g["size"] if g["complete"] else r.size >= g["size"], (i, r.size, g["size"])
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1, i


@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 3)])
def test_restart_small_minimum_batch_equals_oracle(solver, directed, k):
    from paper_1908_06418_b300 import MCS_RESTART
    pairs = _pairs(120, 8, 24, 4500 + k + (50 if directed else 0), directed, k)
    solver.set_restart(32, 5)
    try:
        res = solver.solve_batch(pairs, flags=MCS_RESTART, directed=directed, timeout_s=60)
    finally:
        solver.set_restart(-1, 0)
    for i, (p, r) in enumerate(zip(pairs, res)):
        o = oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed)
        assert r.status == 0 and r.size == o.size, (i, r.size, o.size)
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1, i


def test_restart_lone_searcher(solver):
    """A lone searcher: with a minimum no pair reaches it walks the plain tree
    node for node; with restarts firing its traversal changes (its spilled
    branches come back from the ring in another order) and the optimum does
    not."""
    from paper_1908_06418_b300 import MCS_RESTART, MCS_NO_LEVEL_PRUNE
    pairs = _pairs(16, 12, 18, 4600, pmin=0.3, pmax=0.5)
    solver.set_max_warps(1)
    changed = 0
    try:
        for p in pairs:
            o = oracle.mcs(p.G.adj, p.H.adj)
            solver.set_restart(1 << 50, 0)
            r = solver.solve(p.G.adj, p.H.adj, flags=MCS_RESTART | MCS_NO_LEVEL_PRUNE, timeout_s=30)
            assert r.status == 0 and r.size == o.size and r.nodes == o.nodes
            solver.set_restart(64, 3)
            r = solver.solve(p.G.adj, p.H.adj, flags=MCS_RESTART | MCS_NO_LEVEL_PRUNE, timeout_s=30)
            assert r.status == 0 and r.size == o.size
            assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx) == 1
            changed += r.nodes != o.nodes
    finally:
        solver.set_max_warps(0)
        solver.set_restart(-1, 0)
    assert changed >= len(pairs) // 2


def test_restart_parameters_and_flag_combinations(solver):
    import torch
    from paper_1908_06418_b300 import (MCS_RESTART, MCS_TOP_DOWN, MCS_DEAD_END, MCS_ORDER_LEARNED,
                                       MCS_ERR_ARG, MCS_ERR_UNSUPPORTED, DeviceBatch)
    for bad in (0, -2):
        with pytest.raises(ValueError):
            solver.set_restart(bad, 0)
    pairs = _pairs(4, 6, 10, 4700)
    b = DeviceBatch(pairs)
    n = len(pairs)
    out = [torch.zeros(n, dtype=torch.int32, device=b.device), torch.zeros(n, dtype=torch.int32, device=b.device),
           torch.zeros(n, dtype=torch.int64, device=b.device)]
    for extra, want in ((MCS_TOP_DOWN, MCS_ERR_ARG), (MCS_DEAD_END, MCS_ERR_ARG),
                        (MCS_ORDER_LEARNED, MCS_ERR_UNSUPPORTED)):
        rc = solver.solve_batch_device(n, b.d_n, b.d_adj_off, b.d_adj, b.d_lab_off, b.d_labels, *out,
                                       flags=b.flags | MCS_RESTART | extra, timeout_s=10)
        assert rc == want, (extra, rc)
