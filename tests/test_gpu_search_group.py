"""Searchers narrower than a warp (16, 8, 4 or 2 lanes: two to sixteen independent
depth-first searches per warp) against the CPU oracle: sizes bit-exact,
mappings verified, and a lone searcher walks the oracle's search tree.  Every
test runs in both ways the searchers of a warp can share it: in lockstep (one
predicated node step for all of them per pass) and free-running."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["lockstep", "free"])
def solver(request):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06418_b300 import Solver, MCS_MODE_LOCKSTEP, MCS_MODE_FREE
    s = Solver(0)
    s.set_search_mode(MCS_MODE_LOCKSTEP if request.param == "lockstep" else MCS_MODE_FREE)
    yield s
    s.close()


def _rand_pairs(count, nmin, nmax, seed, directed=False, k=0):
    rs = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nG, nH = int(rs.integers(nmin, nmax + 1)), int(rs.integers(nmin, nmax + 1))
        p = float(rs.uniform(0.1, 0.6))
        rg, rh = synth.rng_for(seed, i, 0), synth.rng_for(seed, i, 1)
        f = synth.er_directed if directed else synth.er_undirected
        out.append(synth.Pair(synth.Graph(f(nG, p, rg), synth.uniform_labels(nG, k, rg)),
                              synth.Graph(f(nH, p, rh), synth.uniform_labels(nH, k, rh)), directed))
    return out


@pytest.fixture
def group(solver, request):
    solver.set_search_group(request.param)
    yield request.param
    solver.set_search_group(32)


@pytest.mark.parametrize("group", [16, 8, 4, 2], indirect=True)
@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 3)])
def test_lone_group_traversal_equals_oracle(solver, group, directed, k):
    from paper_1908_06418_b300 import MCS_NO_LEVEL_PRUNE
    pairs = _rand_pairs(30, 4, 16, 5151 + k + (100 if directed else 0), directed, k)
    solver.set_max_warps(1)
    try:
        for p in pairs:
            r = solver.solve(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed,
                             flags=MCS_NO_LEVEL_PRUNE, timeout_s=30)
            o = oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed)
            assert r.status == 0 and r.size == o.size and r.nodes == o.nodes
            assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1
    finally:
        solver.set_max_warps(0)


@pytest.mark.parametrize("group", [16, 8, 4, 2], indirect=True)
@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 4), (True, 3)])
def test_group_batch_parity(solver, group, directed, k):
    pairs = _rand_pairs(300, 1, 24, 2718 + k + (50 if directed else 0), directed, k)
    res = solver.solve_batch(pairs, directed=directed, timeout_s=60)
    for i, (p, r) in enumerate(zip(pairs, res)):
        o = oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed).size
        assert r.status == 0 and r.size == o, (i, r.status, r.size, o)
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1, i


@pytest.mark.parametrize("group", [8, 4, 2], indirect=True)
def test_group_ragged_sizes_up_to_64(solver, group):
    """Up to 64 classes per node: several slots of an 8-lane group, a ragged last slot."""
    pairs = [synth.Pair(synth.Graph(synth.er_undirected(n, 0.5, synth.rng_for(77, n, 0)),
                                    synth.uniform_labels(n, 20, synth.rng_for(77, n, 2))),
                        synth.Graph(synth.er_undirected(m, 0.5, synth.rng_for(77, n, 1)),
                                    synth.uniform_labels(m, 20, synth.rng_for(77, n, 3))))
             for n, m in [(64, 64), (63, 57), (41, 64), (9, 64), (64, 1), (33, 47)]]
    res = solver.solve_batch(pairs, timeout_s=120)
    for p, r in zip(pairs, res):
        o = oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels)
        assert r.status == 0 and r.size == o.size
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1


@pytest.mark.parametrize("group", [16, 8, 4, 2], indirect=True)
def test_group_learned_order_stays_exact(solver, group):
    from oracle import mlp
    from paper_1908_06418_b300 import MCS_ORDER_LEARNED
    pairs = _rand_pairs(80, 6, 24, 606)
    ref = [oracle.mcs(p.G.adj, p.H.adj).size for p in pairs]
    solver.set_order_model(mlp.init_params(5).astype(np.float32))
    res = solver.solve_batch(pairs, flags=MCS_ORDER_LEARNED, timeout_s=60)
    assert [r.size for r in res] == ref and all(r.status == 0 for r in res)


@pytest.mark.parametrize("group", [8, 4, 2], indirect=True)
def test_group_graph_replay(solver, group):
    import torch
    from paper_1908_06418_b300 import DeviceBatch, MCS_GRAPH_REPLAY
    pairs = _rand_pairs(64, 8, 24, 99)
    ref = np.array([oracle.mcs(p.G.adj, p.H.adj).size for p in pairs])
    b = DeviceBatch(pairs)
    n = len(pairs)
    stream = torch.cuda.Stream(b.device)
    for rep in range(3):
        size = torch.full((n,), -9, dtype=torch.int32, device=b.device)
        status = torch.full((n,), -9, dtype=torch.int32, device=b.device)
        nodes = torch.zeros(n, dtype=torch.int64, device=b.device)
        rc = solver.solve_batch_device(n, b.d_n, b.d_adj_off, b.d_adj, b.d_lab_off, b.d_labels,
                                       size, status, nodes, flags=MCS_GRAPH_REPLAY, timeout_s=60,
                                       stream=stream.cuda_stream)
        stream.synchronize()
        assert rc == 0
        assert (status.cpu().numpy() == 0).all() and (size.cpu().numpy() == ref).all()


def test_invalid_group_is_rejected(solver):
    for bad in (0, 1, 3, 12, 64, -8):
        with pytest.raises(ValueError):
            solver.set_search_group(bad)
    p = synth.config1_pair()
    assert solver.solve(p.G.adj, p.H.adj, timeout_s=10).size == 13
