"""The static component + Hellerman-Rarick-style vertex order (Section IV-A,
MCS_ORDER_HR) on the GPU: the pack kernel must number the vertices as the
oracle's hr_order does (a lone searcher then walks the oracle's tree node for
node), and the optimum must not change."""
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


def _blocks(n, p, rng, directed):
    """A graph of n vertices made of two or three random components (plus an
    isolated vertex or two), randomly renumbered."""
    f = synth.er_directed if directed else synth.er_undirected
    cuts = sorted(rng.choice(np.arange(1, n), size=min(2, n - 1), replace=False).tolist())
    a = np.zeros((n, n), np.uint8)
    lo = 0
    for hi in cuts + [n]:
        m = hi - lo
        if m > 2:
            a[lo:hi, lo:hi] = f(m, p, rng)
        lo = hi
    perm = rng.permutation(n)
    return a[np.ix_(perm, perm)].copy()


def _block_pairs(count, nmin, nmax, seed, directed=False, k=0):
    rs = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nG, nH = int(rs.integers(nmin, nmax + 1)), int(rs.integers(nmin, nmax + 1))
        p = float(rs.uniform(0.25, 0.5))
        rg, rh = synth.rng_for(seed, i, 0), synth.rng_for(seed, i, 1)
        out.append(synth.Pair(synth.Graph(_blocks(nG, p, rg, directed), synth.uniform_labels(nG, k, rg)),
                              synth.Graph(_blocks(nH, p, rh, directed), synth.uniform_labels(nH, k, rh)), directed))
    return out


def _pairs(count, nmin, nmax, seed, directed=False, k=0, pmin=0.08, pmax=0.5):
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


@pytest.mark.parametrize("group", [32, 8])
@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 3)])
def test_hr_order_single_searcher_walks_the_oracle_tree(solver, group, directed, k):
    """Sparse pairs (several components each) and denser ones: equal node
    counts mean the device numbered both graphs exactly as hr_order."""
    from paper_1908_06418_b300 import MCS_ORDER_HR, MCS_NO_LEVEL_PRUNE
    seed = 4100 + k + (50 if directed else 0)
    pairs = _pairs(25, 3, 18, seed, directed, k) + _block_pairs(25, 6, 20, seed + 7, directed, k)
    solver.set_max_warps(1)
    solver.set_search_group(group)
    try:
        for i, p in enumerate(pairs):
            r = solver.solve(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed,
                             flags=MCS_ORDER_HR | MCS_NO_LEVEL_PRUNE, timeout_s=30)
            o = oracle.mcs_hr(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed)
            assert r.status == 0 and o.complete
            assert r.size == o.size, (i, r.size, o.size)
            assert r.nodes == o.nodes, (i, r.nodes, o.nodes)
            assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1
    finally:
        solver.set_max_warps(0)
        solver.set_search_group(8)


def test_hr_order_wide_graphs_walk_the_oracle_tree(solver):
    """33..64 vertices (64-bit rows, vertices in both halves of a lane's
    pair), made of several components."""
    from paper_1908_06418_b300 import MCS_ORDER_HR, MCS_NO_LEVEL_PRUNE
    pairs = _block_pairs(8, 33, 64, 4201, False, 24)
    solver.set_max_warps(1)
    try:
        for i, p in enumerate(pairs):
            r = solver.solve(p.G.adj, p.H.adj, p.G.labels, p.H.labels,
                             flags=MCS_ORDER_HR | MCS_NO_LEVEL_PRUNE, timeout_s=60)
            o = oracle.mcs_hr(p.G.adj, p.H.adj, p.G.labels, p.H.labels)
            assert r.status == 0 and r.size == o.size and r.nodes == o.nodes, (i, r.nodes, o.nodes)
    finally:
        solver.set_max_warps(0)


@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 3)])
def test_hr_order_batch_equals_oracle(solver, directed, k):
    from paper_1908_06418_b300 import MCS_ORDER_HR
    pairs = _pairs(150, 2, 22, 4300 + k + (50 if directed else 0), directed, k)
    res = solver.solve_batch(pairs, flags=MCS_ORDER_HR, directed=directed, timeout_s=60)
    for i, (p, r) in enumerate(zip(pairs, res)):
        o = oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed)
        assert r.status == 0 and r.size == o.size, (i, r.size, o.size)
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1


def test_hr_order_is_not_combined_with_the_learned_order(solver):
    import torch
    from paper_1908_06418_b300 import MCS_ORDER_HR, MCS_ORDER_LEARNED, MCS_ERR_ARG, DeviceBatch
    pairs = _pairs(4, 6, 10, 4400)
    b = DeviceBatch(pairs)
    n = len(pairs)
    out = [torch.zeros(n, dtype=torch.int32, device=b.device), torch.zeros(n, dtype=torch.int32, device=b.device),
           torch.zeros(n, dtype=torch.int64, device=b.device)]
    rc = solver.solve_batch_device(n, b.d_n, b.d_adj_off, b.d_adj, b.d_lab_off, b.d_labels, *out,
                                   flags=b.flags | MCS_ORDER_HR | MCS_ORDER_LEARNED, timeout_s=10)
    assert rc == MCS_ERR_ARG
