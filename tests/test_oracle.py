"""Pins for the CPU oracle against things other than itself: brute force, the
modular-product clique reduction, closed forms, invariants and the paper's
worked example (Table 1, Eq. 1)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_pair(seed, nG, nH, p, directed=False, k=0):
    rg, rh = synth.rng_for(900, seed, 0), synth.rng_for(900, seed, 1)
    f = synth.er_directed if directed else synth.er_undirected
    a, b = f(nG, p, rg), f(nH, p, rh)
    la = synth.uniform_labels(nG, k, rg)
    lb = synth.uniform_labels(nH, k, rh)
    return a, b, la, lb


def _edges(n, e):
    a = np.zeros((n, n), np.uint8)
    for i, j in e:
        a[i, j] = a[j, i] = 1
    return a


def complete(n):
    a = np.ones((n, n), np.uint8)
    np.fill_diagonal(a, 0)
    return a


def path(n):
    return _edges(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n):
    return _edges(n, [(i, (i + 1) % n) for i in range(n)])


# --------------------------------------------------------------------------
# verifier
# --------------------------------------------------------------------------
def test_verifier_hand_cases():
    P3 = path(3)                      # 0-1-2
    K3 = complete(3)
    # identity on the path is valid
    assert oracle.verify(P3, P3, [0, 1, 2], [0, 1, 2]) == 1
    # path into triangle: edge 0-2 missing in P3 but present in K3 -> induced fails
    assert oracle.verify(P3, K3, [0, 1, 2], [0, 1, 2]) == -5
    # two vertices of P3 adjacent map to an edge: fine
    assert oracle.verify(P3, K3, [0, 1], [2, 0]) == 1
    # non-injective
    assert oracle.verify(P3, P3, [0, 1], [1, 1]) == -3
    # out of range
    assert oracle.verify(P3, P3, [0, 3], [1, 2]) == -2
    # labels differ
    assert oracle.verify(P3, P3, [0], [0], np.array([1, 0, 0], np.int32),
                         np.array([0, 0, 0], np.int32)) == -4
    # self-loop on one side only
    L = P3.copy()
    L[1, 1] = 1
    assert oracle.verify(L, P3, [1], [1]) == -6
    # directed: arc only one way
    D = np.zeros((2, 2), np.uint8)
    D[0, 1] = 1
    E = np.zeros((2, 2), np.uint8)
    E[1, 0] = 1
    assert oracle.verify(D, E, [0, 1], [0, 1]) == -5
    assert oracle.verify(D, E, [0, 1], [1, 0]) == 1
    # empty mapping is valid
    assert oracle.verify(P3, K3, [], []) == 1


# --------------------------------------------------------------------------
# brute force (n <= 9) and clique reduction
# --------------------------------------------------------------------------
@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 3), (True, 2)])
def test_oracle_vs_bruteforce(directed, k):
    rs = np.random.default_rng(17 + 31 * k + (1000 if directed else 0))
    for s in range(150):
        nG, nH = int(rs.integers(0, 10)), int(rs.integers(0, 10))
        p = float(rs.uniform(0.1, 0.7))
        a, b, la, lb = _rand_pair(s + (5000 if directed else 0) + 100 * k, nG, nH, p, directed, k)
        r = oracle.mcs(a, b, la, lb, directed=directed)
        kb, bg, bh = oracle.bruteforce(a, b, la, lb)
        assert r.complete
        assert r.size == kb, (s, nG, nH, p)
        assert oracle.verify(a, b, r.g_idx, r.h_idx, la, lb) == 1
        assert oracle.verify(a, b, bg, bh, la, lb) == 1
        assert len(bg) == kb


def test_oracle_vs_bruteforce_selfloops():
    rs = np.random.default_rng(5)
    for s in range(100):
        nG, nH = int(rs.integers(1, 9)), int(rs.integers(1, 9))
        a, b, la, lb = _rand_pair(7000 + s, nG, nH, 0.4, directed=bool(s % 2))
        a[np.diag_indices(nG)] = (rs.random(nG) < 0.3)
        b[np.diag_indices(nH)] = (rs.random(nH) < 0.3)
        r = oracle.mcs(a, b, directed=bool(s % 2))
        assert r.size == oracle.bruteforce(a, b)[0]
        assert oracle.verify(a, b, r.g_idx, r.h_idx) == 1


@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 2)])
def test_oracle_vs_modular_product_clique(directed, k):
    rs = np.random.default_rng(99 + k + (7 if directed else 0))
    for s in range(25):
        nG, nH = int(rs.integers(6, 13)), int(rs.integers(6, 13))
        p = float(rs.uniform(0.15, 0.6))
        a, b, la, lb = _rand_pair(9000 + s + 50 * k + (500 if directed else 0), nG, nH, p,
                                  directed, k)
        r = oracle.mcs(a, b, la, lb, directed=directed)
        kc, cg, ch = oracle.clique(a, b, la, lb)
        assert r.size == kc
        assert oracle.verify(a, b, cg, ch, la, lb) == 1


# --------------------------------------------------------------------------
# closed forms and invariants
# --------------------------------------------------------------------------
def test_closed_forms():
    for a in range(1, 8):
        for b in range(1, 8):
            assert oracle.mcs(complete(a), complete(b)).size == min(a, b)
            assert oracle.mcs(np.zeros((a, a), np.uint8), complete(b)).size == 1
            assert oracle.mcs(path(a), path(b)).size == min(a, b)
    for a in range(3, 9):
        for b in range(a + 1, 11):
            assert oracle.mcs(cycle(a), cycle(b)).size == a - 1
    g = synth.grid(6, 6)
    assert oracle.mcs(g, g).size == 36
    assert oracle.mcs(np.zeros((0, 0), np.uint8), complete(3)).size == 0


def test_closed_forms_beyond_64_vertices():
    """The oracle has no word-size limit; the GPU's multi-word path (65-256
    vertices) is checked against it, so it is pinned at those sizes too:
    paths, cycles, complete and empty graphs, a labelled graph against a
    permuted copy of itself (MCS(G, G) = |V|) and against one of its induced
    subgraphs (MCS = the subgraph's size)."""
    assert oracle.mcs(path(100), path(120)).size == 100
    assert oracle.mcs(cycle(90), cycle(130)).size == 89
    assert oracle.mcs(complete(100), complete(90)).size == 90
    assert oracle.mcs(np.zeros((100, 100), np.uint8), np.zeros((80, 80), np.uint8)).size == 80
    assert oracle.mcs(complete(256), complete(256)).size == 256
    assert oracle.mcs(np.zeros((256, 256), np.uint8), complete(70)).size == 1
    r = synth.rng_for(9102, 0, 0)
    for n, k in ((100, 16), (200, 40), (256, 64)):
        G = synth.er_undirected(n, 0.04, r)
        lab = synth.uniform_labels(n, k, r)
        perm = r.permutation(n)
        res = oracle.mcs(G, G[np.ix_(perm, perm)], lab, lab[perm])
        assert res.complete and res.size == n
        sub = perm[: (2 * n) // 3]
        res = oracle.mcs(G, G[np.ix_(sub, sub)], lab, lab[sub])
        assert res.complete and res.size == len(sub)
        assert oracle.verify(G, G[np.ix_(sub, sub)], res.g_idx, res.h_idx, lab, lab[sub]) == 1


def test_invariants():
    rs = np.random.default_rng(3)
    for s in range(40):
        directed = bool(s % 2)
        n1, n2 = int(rs.integers(5, 15)), int(rs.integers(5, 15))
        a, b, _, _ = _rand_pair(12000 + s, n1, n2, float(rs.uniform(0.1, 0.5)), directed)
        k = oracle.mcs(a, b, directed=directed).size
        assert oracle.mcs(a, a, directed=directed).size == n1            # MCS(G,G) = |V|
        assert oracle.mcs(b, a, directed=directed).size == k             # symmetry
        perm = rs.permutation(n2)
        assert oracle.mcs(a, b[np.ix_(perm, perm)], directed=directed).size == k
        perm = rs.permutation(n1)
        assert oracle.mcs(a[np.ix_(perm, perm)], b, directed=directed).size == k
        assert 1 <= k <= min(n1, n2)
        if not directed:                                                  # complements
            ca, cb = 1 - a, 1 - b
            np.fill_diagonal(ca, 0)
            np.fill_diagonal(cb, 0)
            assert oracle.mcs(ca, cb).size == k


def test_planted_core_lower_bound():
    for s in range(6):
        rng = synth.rng_for(77, s, 0)
        p = synth.planted_pair(16, 0.5, 0.3, rng)
        assert oracle.mcs(p.G.adj, p.H.adj).size >= 8


def test_labels_restrict():
    # identical graphs but labels that disagree everywhere: nothing matches
    a = complete(5)
    assert oracle.mcs(a, a, np.zeros(5, np.int32), np.ones(5, np.int32)).size == 0
    la = np.array([0, 0, 1, 1, 2], np.int32)
    assert oracle.mcs(a, a, la, la).size == 5


# --------------------------------------------------------------------------
# worked example (Table 1) and Eq. 1
# --------------------------------------------------------------------------
def test_table1_split_and_bound():
    fx = json.load(open(os.path.join(HERE, "golden", "table1.json")))
    G = _edges(4, fx["G_edges"])
    H = _edges(4, fx["H_edges"])
    bounds, cg, ch = oracle.split_trace(G, H, fx["mapping_g"], fx["mapping_h"])
    assert list(bounds) == fx["bound_after_step_eq1"]
    for t, lab in enumerate(fx["labels_after_step"]):
        lg = {int(k): v for k, v in lab["G"].items()}
        lh = {int(k): v for k, v in lab["H"].items()}
        common = set(lg.values()) & set(lh.values())
        # same label string on both sides <=> same class; a label present on one
        # side only gives no class (its vertices can never be matched)
        for x in range(4):
            if x in lg and lg[x] in common:
                for y in range(4):
                    if y in lh:
                        assert (cg[t, x] == ch[t, y]) == (lg[x] == lh[y])
            else:
                assert cg[t, x] == -1
        for y in range(4):
            if not (y in lh and lh[y] in common):
                assert ch[t, y] == -1


def test_node_counts_tiny_hand_derived():
    # K1 vs K1: root, child (0,0) pruned at its bound (=1 <= incumbent 1),
    # then the unmatched-v node with no classes: 3 calls.
    assert oracle.mcs(complete(1), complete(1)).nodes == 3
    # K2 vs K2 worked by hand under the bound <= incumbent rule: 6 calls.
    assert oracle.mcs(complete(2), complete(2)).nodes == 6


def test_node_limit_gives_lower_bound():
    p = synth.config1_pair()
    r = oracle.mcs(p.G.adj, p.H.adj, node_limit=500)
    assert not r.complete
    assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx) == 1
    assert r.size <= 13


def test_config1_golden_matches_generator():
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    from make_oracle_golden import pair_digest
    rows = [json.loads(x) for x in open(os.path.join(HERE, "golden", "c1_oracle.jsonl"))]
    p = synth.config1_pair()
    assert rows[0]["digest"] == pair_digest(p)
    assert rows[0]["size"] == oracle.mcs(p.G.adj, p.H.adj).size == 13


# --------------------------------------------------------------------------
# goal-directed search and the top-down strategy (Section IV-A)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 3), (True, 2)])
def test_topdown_vs_bruteforce(directed, k):
    """Top-down reaches the same optimum as exhaustive enumeration (a
    different traversal: goal searches from min(|V_G|,|V_H|) down)."""
    rs = np.random.default_rng(61 + 7 * k + (500 if directed else 0))
    for s in range(120):
        nG, nH = int(rs.integers(0, 10)), int(rs.integers(0, 10))
        p = float(rs.uniform(0.1, 0.7))
        a, b, la, lb = _rand_pair(s + 7000 + (5000 if directed else 0) + 100 * k, nG, nH, p, directed, k)
        r = oracle.mcs_topdown(a, b, la, lb, directed=directed)
        kb, _, _ = oracle.bruteforce(a, b, la, lb)
        assert r.complete
        assert r.size == kb, (s, nG, nH, p)
        assert len(r.g_idx) == r.size
        assert oracle.verify(a, b, r.g_idx, r.h_idx, la, lb) == 1


@pytest.mark.parametrize("directed,k", [(False, 0), (True, 2)])
def test_goal_search_decides_each_goal(directed, k):
    """A goal search with floor g-1 and cap g records a mapping (of size
    exactly g) iff a common induced subgraph of g vertices exists, i.e. iff
    the optimum found by exhaustive enumeration is >= g."""
    rs = np.random.default_rng(83 + k)
    for s in range(40):
        nG, nH = int(rs.integers(1, 9)), int(rs.integers(1, 9))
        a, b, la, lb = _rand_pair(s + 8000 + 100 * k, nG, nH, float(rs.uniform(0.2, 0.6)), directed, k)
        opt, _, _ = oracle.bruteforce(a, b, la, lb)
        for goal in range(1, min(nG, nH) + 2):
            r = oracle.mcs_goal(a, b, goal - 1, goal, la, lb, directed=directed)
            assert r.complete
            if opt >= goal:
                assert r.size == goal, (s, goal, opt)
                assert oracle.verify(a, b, r.g_idx, r.h_idx, la, lb) == 1
            else:
                assert r.size == 0, (s, goal, opt)


def test_topdown_on_an_induced_subgraph_stops_at_the_first_goal():
    """When G is an induced subgraph of H the first goal, |V_G|, is reached:
    top-down is exactly one goal search, and it maps all of G."""
    rs = np.random.default_rng(97)
    for s in range(20):
        n = int(rs.integers(6, 16))
        _, b, _, _ = _rand_pair(s + 9000, n, n + 6, 0.35)
        keep = np.sort(rs.permutation(n + 6)[:n])
        a = b[np.ix_(keep, keep)].copy()
        r = oracle.mcs_topdown(a, b)
        one = oracle.mcs_goal(a, b, n - 1, n)
        assert r.size == n and one.size == n
        assert r.nodes == one.nodes
        assert oracle.verify(a, b, r.g_idx, r.h_idx) == 1


def test_topdown_nodes_sum_over_goal_searches():
    """Top-down's node count is the sum over the goal searches it ran, from
    min(|V_G|,|V_H|) down to the optimum."""
    for s in range(12):
        a, b, _, _ = _rand_pair(s + 9500, 11, 13, 0.4)
        r = oracle.mcs_topdown(a, b)
        opt = oracle.mcs(a, b).size
        assert r.size == opt
        total = sum(oracle.mcs_goal(a, b, g - 1, g).nodes for g in range(11, opt - 1, -1))
        assert r.nodes == total


@pytest.mark.parametrize("threshold,doubling", [(1, False), (3, False), (20, False), (1, True), (7, True)])
def test_deadend_vs_bruteforce(threshold, doubling):
    """Dead-end forecasting reaches the optimum of exhaustive enumeration
    whatever the threshold: raised bounds that are unreachable are closed by
    the binary search, reachable ones are overtaken by a larger mapping."""
    rs = np.random.default_rng(131 + threshold + (50 if doubling else 0))
    for s in range(80):
        directed = bool(s % 3 == 0)
        k = 3 if s % 4 == 1 else 0
        nG, nH = int(rs.integers(0, 10)), int(rs.integers(0, 10))
        a, b, la, lb = _rand_pair(s + 10000 + 97 * threshold, nG, nH, float(rs.uniform(0.1, 0.7)), directed, k)
        r = oracle.mcs_deadend(a, b, threshold, doubling, la, lb, directed=directed)
        kb, _, _ = oracle.bruteforce(a, b, la, lb)
        assert r.complete
        assert r.size == kb, (s, threshold, doubling, r.size, kb)
        assert len(r.g_idx) == r.size
        assert oracle.verify(a, b, r.g_idx, r.h_idx, la, lb) == 1


def test_deadend_with_a_huge_threshold_is_the_plain_search():
    """A threshold that is never reached leaves the plain search unchanged,
    node for node."""
    for s in range(15):
        a, b, _, _ = _rand_pair(s + 11000, 12, 14, 0.4)
        r = oracle.mcs_deadend(a, b, 1 << 40)
        o = oracle.mcs(a, b)
        assert r.size == o.size and r.nodes == o.nodes


def test_deadend_raises_change_the_traversal_on_larger_pairs():
    """On pairs whose plain search runs long after its last improvement, a
    small threshold raises the bound (the traversal differs from the plain
    one) and the optimum is unchanged."""
    changed = 0
    for s in range(10):
        a, b, _, _ = _rand_pair(s + 12000, 16, 18, 0.5)
        o = oracle.mcs(a, b)
        r = oracle.mcs_deadend(a, b, 50)
        assert r.size == o.size
        changed += r.nodes != o.nodes
    assert changed >= 5


# --------------------------------------------------------------------------
# static component + Hellerman-Rarick-style order (Section IV-A)
# --------------------------------------------------------------------------
def test_hr_order_hand_derived_cases():
    """Orders derived by hand from the procedure of Section IV-A (components
    by decreasing rows/columns ratio, then size; inside a component the
    column meeting most of the shortest active rows goes next):
    path 0-1-2-3-4: shortest rows {0,4} -> column 1 (tie with 3, lower
    first); then rows {2,4} -> 3; then rows {1,3} -> 2; then 0, 4.
    star 0-{1,2,3,4}, edge 6-7, isolated 5: the star (ratio 1, size 5), its
    centre first; then the edge; the isolated vertex (ratio 0) last.
    triangle 0-1-2 beside the 4-cycle 3-4-5-6: the larger component first,
    3 (all rows tie), then 5 (meets both shortest rows 4 and 6), 4, 6.
    arcs 0->1->2 and 3->4, vertex 5: columns are in-arcs, so 1, 2, then the
    vertex without an in-arc, 0."""
    def E(n, edges):
        a = np.zeros((n, n), np.uint8)
        for i, j in edges:
            a[i, j] = a[j, i] = 1
        return a
    assert oracle.hr_order(E(5, [(0, 1), (1, 2), (2, 3), (3, 4)])).tolist() == [1, 3, 2, 0, 4]
    assert oracle.hr_order(E(8, [(0, 1), (0, 2), (0, 3), (0, 4), (6, 7)])).tolist() == [0, 1, 2, 3, 4, 6, 7, 5]
    assert oracle.hr_order(E(7, [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (5, 6), (6, 3)])).tolist() == \
        [3, 5, 4, 6, 0, 1, 2]
    d = np.zeros((6, 6), np.uint8)
    d[0, 1] = d[1, 2] = d[3, 4] = 1
    assert oracle.hr_order(d, directed=True).tolist() == [1, 2, 0, 4, 3, 5]


def test_hr_order_is_a_permutation_with_contiguous_components():
    rs = np.random.default_rng(141)
    for s in range(60):
        n = int(rs.integers(1, 40))
        directed = bool(s % 2)
        f = synth.er_directed if directed else synth.er_undirected
        a = f(n, float(rs.uniform(0.02, 0.3)), synth.rng_for(141, s, 0))
        perm = oracle.hr_order(a, directed=directed)
        assert sorted(perm.tolist()) == list(range(n))
        und = ((a | a.T) != 0).astype(np.int64)
        np.fill_diagonal(und, 0)
        # component label of each vertex (closure by repeated squaring)
        reach = (und + np.eye(n, dtype=np.int64)) > 0
        for _ in range(7):
            reach = (reach.astype(np.int64) @ reach.astype(np.int64)) > 0
        lab = [int(np.argmax(reach[x])) for x in range(n)]
        seq = [lab[x] for x in perm]
        seen = set()
        for i, c in enumerate(seq):
            if i and c != seq[i - 1]:
                assert c not in seen, (s, seq)
            seen.add(c)


@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 3)])
def test_mcs_with_hr_order_vs_bruteforce(directed, k):
    """The order changes the traversal only: the optimum is enumeration's."""
    rs = np.random.default_rng(151 + k + (7 if directed else 0))
    for s in range(100):
        nG, nH = int(rs.integers(0, 10)), int(rs.integers(0, 10))
        a, b, la, lb = _rand_pair(s + 13000 + 100 * k, nG, nH, float(rs.uniform(0.1, 0.7)), directed, k)
        r = oracle.mcs_hr(a, b, la, lb, directed=directed)
        kb, _, _ = oracle.bruteforce(a, b, la, lb)
        assert r.complete and r.size == kb
        assert oracle.verify(a, b, r.g_idx, r.h_idx, la, lb) == 1


# --------------------------------------------------------------------------
# randomized restarts over an explicit stack of pending branches (Section IV-A)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("directed,k", [(False, 0), (True, 0), (False, 3)])
def test_restart_stack_without_restarts_is_the_recursion(directed, k):
    """With no restart firing, the explicit stack walks the recursive
    search's tree node for node."""
    rs = np.random.default_rng(171 + k)
    for s in range(30):
        nG, nH = int(rs.integers(0, 15)), int(rs.integers(0, 15))
        a, b, la, lb = _rand_pair(s + 14000 + 100 * k, nG, nH, float(rs.uniform(0.1, 0.6)), directed, k)
        r, n = oracle.mcs_restart(a, b, 1 << 60, 0, la, lb, directed=directed)
        o = oracle.mcs(a, b, la, lb, directed=directed)
        assert n == 0 and r.size == o.size and r.nodes == o.nodes


@pytest.mark.parametrize("min_nodes,seed", [(1, 0), (1, 12345), (8, 7), (64, 99)])
def test_restart_vs_bruteforce(min_nodes, seed):
    """Restarts reorder the pending branches, which hold every part of the
    tree not yet visited: the optimum is enumeration's for any seed."""
    rs = np.random.default_rng(181 + min_nodes + seed % 1000)
    total = 0
    for s in range(80):
        directed = bool(s % 3 == 0)
        k = 3 if s % 4 == 1 else 0
        nG, nH = int(rs.integers(0, 10)), int(rs.integers(0, 10))
        a, b, la, lb = _rand_pair(s + 15000 + min_nodes, nG, nH, float(rs.uniform(0.1, 0.7)), directed, k)
        r, n = oracle.mcs_restart(a, b, min_nodes, seed, la, lb, directed=directed)
        kb, _, _ = oracle.bruteforce(a, b, la, lb)
        assert r.complete and r.size == kb, (s, r.size, kb)
        assert oracle.verify(a, b, r.g_idx, r.h_idx, la, lb) == 1
        total += n
    assert total > 0


def test_restarts_fire_and_keep_the_optimum_on_larger_pairs():
    fired = 0
    for s in range(10):
        a, b, _, _ = _rand_pair(s + 16000, 16, 18, 0.5)
        o = oracle.mcs(a, b)
        r, n = oracle.mcs_restart(a, b, 256, s)
        assert r.size == o.size
        fired += n > 0
    assert fired >= 5
