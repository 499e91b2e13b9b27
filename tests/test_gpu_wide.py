"""Graphs of 65 to 256 vertices: the multi-word path (two words per vertex set
up to 128 vertices, four up to 256) against the CPU oracle.

Random pairs of this size are beyond the oracle (the paper itself solves no
pair above 50 vertices within 1,000 s), so the pairs here have structure that
keeps the proof short: a graph against a permuted copy of itself with a few
arcs flipped (labelled and unlabelled, undirected and directed), an induced
subgraph of a graph against the graph, paths, cycles, complete and empty
graphs.  Sizes are compared bit-exactly, mappings verified, and a lone
searcher must visit exactly the oracle's nodes (the same class choice and
candidate order on multi-word bit sets)."""
import numpy as np
import pytest

import oracle
import synth
from paper_1908_06418_b300 import MCS_MAX_N

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


def _perturbed_pairs(count, seed, nmin, nmax, p_range, k_range, flips, directed=False):
    """G(n, p) against a random permutation of itself with `flips` arcs
    toggled: the optimum is near n, and the proof stays short."""
    out = []
    for i in range(count):
        r = synth.rng_for(seed, i, 0)
        n = int(r.integers(nmin, nmax + 1))
        p = float(r.uniform(*p_range))
        k = int(r.integers(k_range[0], k_range[1] + 1))
        G = (synth.er_directed if directed else synth.er_undirected)(n, p, r)
        lab = synth.uniform_labels(n, k, r) if k else None
        H = G.copy()
        for _ in range(flips):
            a, b = (int(x) for x in r.integers(0, n, 2))
            if a == b:
                continue
            H[a, b] ^= 1
            if not directed:
                H[b, a] = H[a, b]
        perm = r.permutation(n)
        H = H[np.ix_(perm, perm)]
        lh = None if lab is None else lab[perm]
        out.append(synth.Pair(synth.Graph(G, lab), synth.Graph(H, lh), directed, f"pert-{seed}-{i}"))
    return out


def _closed_forms():
    """(pair, optimum) with the optimum known in closed form."""
    def path(n):
        a = np.zeros((n, n), np.uint8)
        for i in range(n - 1):
            a[i, i + 1] = a[i + 1, i] = 1
        return a

    def cycle(n):
        a = path(n)
        a[0, n - 1] = a[n - 1, 0] = 1
        return a

    K = lambda n: (np.ones((n, n), np.uint8) - np.eye(n, dtype=np.uint8))
    E = lambda n: np.zeros((n, n), np.uint8)
    r = synth.rng_for(9101, 0, 0)
    G = synth.er_undirected(180, 0.03, r)
    lab = synth.uniform_labels(180, 40, r)
    sub = r.permutation(180)[:120]
    cases = [(path(100), path(120), None, None, 100), (cycle(90), cycle(130), None, None, 89),
             (K(100), K(90), None, None, 90), (E(100), E(80), None, None, 80), (K(256), K(256), None, None, 256),
             (E(256), K(70), None, None, 1), (G, G[np.ix_(sub, sub)], lab, lab[sub], 120)]
    return [(synth.Pair(synth.Graph(a, la), synth.Graph(b, lb), False), k) for a, b, la, lb, k in cases]


def _check(pairs, res, want=None):
    for i, (p, r) in enumerate(zip(pairs, res)):
        o = oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=p.directed) if want is None else None
        k = want[i] if want is not None else o.size
        if want is None:
            assert o.complete, i
        assert r.status == 0, (i, r.status)
        assert r.size == k, (i, r.size, k)
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1, i


@pytest.mark.parametrize("case", ["undirected", "labelled-few", "labelled", "directed", "labelled-256"])
def test_wide_single_searcher_walks_the_oracle_tree(solver, case):
    """One searcher, no level prune: the device visits exactly the oracle's
    nodes on graphs of 65-128 vertices (two words) and 129-256 (four)."""
    from paper_1908_06418_b300 import MCS_NO_LEVEL_PRUNE
    if case == "undirected":
        # unlabelled: paths, cycles, complete and empty graphs (two and four words)
        pairs = [p for p, _ in _closed_forms()[:6]]
    elif case == "labelled-few":
        pairs = _perturbed_pairs(8, 7101, 65, 100, (0.1, 0.2), (2, 3), 2)
    elif case == "labelled":
        pairs = _perturbed_pairs(10, 7102, 65, 128, (0.05, 0.1), (6, 10), 4)
    elif case == "directed":
        pairs = _perturbed_pairs(10, 7103, 65, 110, (0.04, 0.08), (6, 10), 4, directed=True)
    else:
        pairs = _perturbed_pairs(8, 7104, 129, 256, (0.02, 0.04), (24, 40), 3)
    solver.set_max_warps(1)
    try:
        for i, p in enumerate(pairs):
            o = oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=p.directed, time_limit_s=60)
            if not o.complete or o.nodes > 3_000_000:
                continue                         # keep the lone searcher's work small
            r = solver.solve(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=p.directed,
                             flags=MCS_NO_LEVEL_PRUNE, timeout_s=120)
            assert r.status == 0 and r.size == o.size, (i, r.status, r.size, o.size)
            assert r.nodes == o.nodes, (i, r.nodes, o.nodes)
            assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1
    finally:
        solver.set_max_warps(0)


def test_wide_batch_parity_with_mixed_sizes(solver):
    """One mcs_solve_batch call with pairs of 8-64 vertices (one-word launch)
    and of 65-256 vertices (multi-word launch) interleaved: every size equals
    the oracle's, every mapping verifies, results come back in call order."""
    small = [synth.Pair(synth.Graph(synth.er_undirected(n, 0.3, synth.rng_for(7200, n, 0)),
                                    synth.uniform_labels(n, 3, synth.rng_for(7200, n, 0))),
                        synth.Graph(synth.er_undirected(n + 3, 0.3, synth.rng_for(7200, n, 1)),
                                    synth.uniform_labels(n + 3, 3, synth.rng_for(7200, n, 1))))
             for n in range(8, 40, 2)]
    wide = (_perturbed_pairs(24, 7201, 65, 128, (0.05, 0.1), (6, 10), 3) +
            _perturbed_pairs(12, 7202, 129, 256, (0.02, 0.04), (24, 40), 2))
    pairs = []
    for i in range(max(len(small), len(wide))):
        if i < len(wide):
            pairs.append(wide[i])
        if i < len(small):
            pairs.append(small[i])
    res = solver.solve_batch(pairs, timeout_s=120)
    _check(pairs, res)


def test_wide_directed_batch(solver):
    pairs = _perturbed_pairs(24, 7203, 65, 128, (0.03, 0.08), (6, 12), 4, directed=True)
    res = solver.solve_batch(pairs, directed=True, timeout_s=120)
    _check(pairs, res)


def test_wide_closed_forms(solver):
    cases = _closed_forms()
    pairs = [p for p, _ in cases]
    res = solver.solve_batch(pairs, timeout_s=120)
    _check(pairs, res, [k for _, k in cases])


def test_wide_device_entry_point(solver):
    """mcs_solve_batch_device with MCS_WIDE (four words, class stacks sized
    for 256 vertices): sizes as the oracle's, mappings at stride MCS_MAX_N."""
    import torch
    from paper_1908_06418_b300 import DeviceBatch, MCS_WIDE
    pairs = _perturbed_pairs(16, 7205, 65, 200, (0.03, 0.08), (12, 20), 2)
    b = DeviceBatch(pairs)
    assert b.flags & MCS_WIDE
    n = len(pairs)
    size = torch.zeros(n, dtype=torch.int32, device=b.device)
    status = torch.zeros(n, dtype=torch.int32, device=b.device)
    nodes = torch.zeros(n, dtype=torch.int64, device=b.device)
    mp = torch.zeros(n * MCS_MAX_N, dtype=torch.int16, device=b.device)
    solver.set_max_warps(256)
    try:
        rc = solver.solve_batch_device(n, b.d_n, b.d_adj_off, b.d_adj, b.d_lab_off, b.d_labels, size, status,
                                       nodes, mp, flags=b.flags, timeout_s=120)
        torch.cuda.synchronize()
    finally:
        solver.set_max_warps(0)
    assert rc == 0
    sz, st = size.cpu().numpy(), status.cpu().numpy()
    mp = mp.cpu().numpy().reshape(n, MCS_MAX_N)
    for i, p in enumerate(pairs):
        o = oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels)
        assert o.complete and st[i] == 0 and sz[i] == o.size, (i, st[i], sz[i], o.size)
        g = np.nonzero(mp[i] >= 0)[0]
        assert len(g) == sz[i]
        assert oracle.verify(p.G.adj, p.H.adj, g, mp[i][g], p.G.labels, p.H.labels) == 1


def test_wide_time_limit_reports_a_verified_lower_bound(solver):
    """A random pair of 200 vertices cannot be proven: a 0.3 s limit ends it
    with MCS_TIMEOUT and a verified mapping."""
    from paper_1908_06418_b300 import MCS_TIMEOUT
    r0 = synth.rng_for(7205, 0, 0)
    G, H = synth.er_undirected(200, 0.2, r0), synth.er_undirected(190, 0.2, synth.rng_for(7205, 0, 1))
    r = solver.solve(G, H, timeout_s=0.3)
    assert r.status == MCS_TIMEOUT
    assert r.size > 0 and oracle.verify(G, H, r.g_idx, r.h_idx) == 1


def test_wide_limits_and_unsupported_options(solver):
    """More than MCS_MAX_N vertices is MCS_ERR_ARG; options of the one-word
    path only (learned order, static order, top-down) are MCS_ERR_UNSUPPORTED
    for pairs over 64 vertices and do not affect the others in the call;
    serving takes graphs of up to 64 vertices."""
    from paper_1908_06418_b300 import (MCS_ERR_ARG, MCS_ERR_UNSUPPORTED, MCS_TOP_DOWN, MCS_ORDER_HR)
    big = np.zeros((MCS_MAX_N + 1, MCS_MAX_N + 1), np.uint8)
    r = solver.solve_batch([(big, big[:10, :10], None, None)], raise_errors=False)[0]
    assert r.status == MCS_ERR_ARG
    wide = _perturbed_pairs(1, 7206, 70, 80, (0.05, 0.1), (6, 6), 2)[0]
    small = synth.Pair(synth.Graph(synth.er_undirected(12, 0.3, synth.rng_for(7206, 1, 0))),
                       synth.Graph(synth.er_undirected(14, 0.3, synth.rng_for(7206, 1, 1))))
    for flags in (MCS_TOP_DOWN, MCS_ORDER_HR):
        res = solver.solve_batch([wide, small], flags=flags, timeout_s=60, raise_errors=False)
        assert res[0].status == MCS_ERR_UNSUPPORTED
        assert res[1].status == 0 and res[1].size == oracle.mcs(small.G.adj, small.H.adj).size
    with pytest.raises(RuntimeError):
        solver.submit(wide.G.adj, wide.H.adj, wide.G.labels, wide.H.labels)
