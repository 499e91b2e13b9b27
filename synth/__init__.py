"""Seeded synthetic graph-pair generators.

This module only draws random graphs.  It holds none of the search method's
arithmetic, so both the CPU oracle (``oracle/``) and the CUDA path
(``paper_1908_06418_b300``) can be fed from it without sharing any code of the
method itself.

Every graph is an ``n x n`` ``uint8`` adjacency matrix, row major, with
``adj[i, j] == 1`` iff there is an edge (arc) ``i -> j``; undirected graphs are
symmetric.  Labels are ``int32`` arrays of length ``n`` or ``None`` (unlabelled).
No generator emits self-loops.

The paper measures on the ARG database's ``mcs10``..``mcs90`` pairs (bounded
valence graphs and 2D/3D/4D meshes, Section V-A); that database is not
available here, so the families below (Erdos-Renyi, random regular, perturbed
meshes and grids) stand in for it.  Seeds follow one rule everywhere:
``Generator(PCG64(SeedSequence([config_id, pair_idx, side])))``.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Iterator, List, Optional

import numpy as np

__all__ = [
    "Graph", "Pair", "rng_for", "er_undirected", "er_directed", "grid",
    "delete_edges", "random_regular", "perturbed_mesh", "uniform_labels",
    "config1_pair", "config2_pairs", "config3_pairs", "config4_pairs",
    "config4_train_pairs", "config5_requests", "planted_pair",
]


@dataclass
class Graph:
    adj: np.ndarray                   # uint8 [n, n]
    labels: Optional[np.ndarray] = None   # int32 [n] or None

    @property
    def n(self) -> int:
        return int(self.adj.shape[0])


@dataclass
class Pair:
    G: Graph
    H: Graph
    directed: bool = False
    tag: str = ""


def rng_for(config_id: int, pair_idx: int, side: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(
        np.random.SeedSequence([int(config_id), int(pair_idx), int(side)])))


# --------------------------------------------------------------------------
# graph families
# --------------------------------------------------------------------------
def er_undirected(n: int, p: float, rng: np.random.Generator) -> np.ndarray:
    """G(n, p): each unordered pair {i, j}, i < j, is an edge independently."""
    a = np.zeros((n, n), dtype=np.uint8)
    if n > 1:
        iu, ju = np.triu_indices(n, 1)
        keep = rng.random(iu.size) < p
        a[iu[keep], ju[keep]] = 1
        a[ju[keep], iu[keep]] = 1
    return a


def er_directed(n: int, p: float, rng: np.random.Generator) -> np.ndarray:
    """Directed G(n, p): each ordered pair (i, j), i != j, is an arc independently."""
    a = (rng.random((n, n)) < p).astype(np.uint8)
    np.fill_diagonal(a, 0)
    return a


def grid(w: int, h: int) -> np.ndarray:
    """Undirected w x h 2D grid; vertex (x, y) has index y * w + x."""
    n = w * h
    a = np.zeros((n, n), dtype=np.uint8)
    for y in range(h):
        for x in range(w):
            i = y * w + x
            if x + 1 < w:
                a[i, i + 1] = a[i + 1, i] = 1
            if y + 1 < h:
                a[i, i + w] = a[i + w, i] = 1
    return a


def _edge_list(a: np.ndarray) -> np.ndarray:
    iu, ju = np.nonzero(np.triu(a, 1))
    return np.stack([iu, ju], axis=1)


def delete_edges(a: np.ndarray, k: int, rng: np.random.Generator) -> np.ndarray:
    """Remove k distinct undirected edges chosen uniformly."""
    a = a.copy()
    e = _edge_list(a)
    k = min(k, len(e))
    pick = rng.choice(len(e), size=k, replace=False) if k else []
    for t in pick:
        i, j = e[t]
        a[i, j] = a[j, i] = 0
    return a


def add_edges(a: np.ndarray, k: int, rng: np.random.Generator) -> np.ndarray:
    """Add k distinct undirected non-edges chosen uniformly (no self-loops)."""
    a = a.copy()
    n = a.shape[0]
    iu, ju = np.triu_indices(n, 1)
    free = np.nonzero(a[iu, ju] == 0)[0]
    k = min(k, free.size)
    pick = rng.choice(free.size, size=k, replace=False) if k else []
    for t in pick:
        i, j = iu[free[t]], ju[free[t]]
        a[i, j] = a[j, i] = 1
    return a


def random_regular(n: int, d: int, rng: np.random.Generator,
                   max_tries: int = 10000) -> np.ndarray:
    """Random d-regular simple graph by the pairing (configuration) model with
    rejection of loops and multi-edges.  Requires n * d even."""
    if (n * d) % 2:
        raise ValueError("n * d must be even")
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n), d)
        rng.shuffle(stubs)
        u, v = stubs[0::2], stubs[1::2]
        if np.any(u == v):
            continue
        a = np.zeros((n, n), dtype=np.uint8)
        ok = True
        for x, y in zip(u, v):
            if a[x, y]:
                ok = False
                break
            a[x, y] = a[y, x] = 1
        if ok:
            return a
    raise RuntimeError("random_regular: too many rejections")


def perturbed_mesh(w: int, h: int, rng: np.random.Generator,
                   frac: float = 0.1) -> np.ndarray:
    """w x h 2D mesh; round(frac * |E|) edges deleted and as many non-edges added."""
    a = grid(w, h)
    k = int(round(frac * len(_edge_list(a))))
    a = delete_edges(a, k, rng)
    return add_edges(a, k, rng)


def uniform_labels(n: int, k: int, rng: np.random.Generator) -> Optional[np.ndarray]:
    """k == 0 means unlabelled; otherwise labels uniform in [0, k)."""
    if k <= 0:
        return None
    return rng.integers(0, k, size=n).astype(np.int32)


def _permute(a: np.ndarray, labels, rng):
    perm = rng.permutation(a.shape[0])
    a2 = a[np.ix_(perm, perm)]
    return a2, (None if labels is None else labels[perm])


# --------------------------------------------------------------------------
# workload configurations
# --------------------------------------------------------------------------
def config1_pair() -> Pair:
    """One pair of undirected unlabelled G(20, 0.3), seeds (1,0,0) and (1,0,1)."""
    return Pair(Graph(er_undirected(20, 0.3, rng_for(1, 0, 0))),
                Graph(er_undirected(20, 0.3, rng_for(1, 0, 1))), False, "c1")


def config1_like(count: int, n: int = 20, p: float = 0.3, cid: int = 11) -> List[Pair]:
    """More pairs of the same family as config 1 (distinct config id)."""
    return [Pair(Graph(er_undirected(n, p, rng_for(cid, i, 0))),
                 Graph(er_undirected(n, p, rng_for(cid, i, 1))), False, f"c1x{i}")
            for i in range(count)]


def config2_pairs(seeds: int = 32, n: int = 36, ps=(0.05, 0.1, 0.3),
                  with_grid: bool = True, cid: int = 2) -> List[Pair]:
    """Directed unlabelled G(n, p) pairs, ``seeds`` per p, plus one pair of
    undirected 6x6 grids each losing round(0.1 * 60) = 6 random edges."""
    out = []
    idx = 0
    for p in ps:
        for s in range(seeds):
            out.append(Pair(Graph(er_directed(n, p, rng_for(cid, idx, 0))),
                            Graph(er_directed(n, p, rng_for(cid, idx, 1))),
                            True, f"c2-p{p}-s{s}"))
            idx += 1
    if with_grid:
        g = grid(6, 6)
        out.append(Pair(Graph(delete_edges(g, 6, rng_for(cid, 1000, 0))),
                        Graph(delete_edges(g, 6, rng_for(cid, 1000, 1))),
                        False, "c2-grid6x6"))
    return out


def shard_cid(cid: int, shard: int) -> int:
    """Config id of a workload's shard: shard 0 is the workload itself; shard
    r > 0 draws the same recipe from seeds of its own (config ids from
    100,000 up, disjoint from every other generator's)."""
    return cid if shard == 0 else 100000 + 1000 * int(shard) + int(cid)


def config3_pairs(count: int = 4096, nmin: int = 10, nmax: int = 40,
                  pmin: float = 0.05, pmax: float = 0.4, k: int = 4,
                  cid: int = 3) -> List[Pair]:
    """Undirected labelled pairs; n_G, n_H independent U{nmin..nmax}, p per
    graph U[pmin, pmax], labels uniform in [0, k)."""
    out = []
    for i in range(count):
        gs = []
        for side in (0, 1):
            r = rng_for(cid, i, side)
            n = int(r.integers(nmin, nmax + 1))
            p = float(r.uniform(pmin, pmax))
            a = er_undirected(n, p, r)
            gs.append(Graph(a, uniform_labels(n, k, r)))
        out.append(Pair(gs[0], gs[1], False, f"c3-{i}"))
    return out


def _c4_graph(r: np.random.Generator, nmin: int, nmax: int, family: int) -> np.ndarray:
    if family == 0:
        d = int(r.integers(3, 5))
        n = int(r.integers(nmin, nmax + 1))
        if (n * d) % 2:
            n += 1 if n + 1 <= nmax else -1
        return random_regular(n, d, r)
    # perturbed 2D mesh with w*h in [nmin, nmax]
    shapes = [(w, h) for w in range(2, nmax + 1) for h in range(w, nmax + 1)
              if nmin <= w * h <= nmax and w >= 3]
    w, h = shapes[int(r.integers(0, len(shapes)))]
    return perturbed_mesh(w, h, r)


def config4_pair(i: int, nmin: int = 40, nmax: int = 64, cid: int = 4) -> Pair:
    """Pair i of the bounded-valence family: even i random 3-/4-regular, odd
    i perturbed 2D meshes (10% edges deleted, as many added)."""
    fam = i % 2
    gs = [_c4_graph(rng_for(cid, i, s), nmin, nmax, fam) for s in (0, 1)]
    return Pair(Graph(gs[0]), Graph(gs[1]), False, f"c4-{cid}-{i}")


def config4_pairs(count: int = 2048, nmin: int = 40, nmax: int = 64,
                  cid: int = 4) -> List[Pair]:
    """Bounded-valence pairs: half random 3-/4-regular, half perturbed 2D
    meshes (10% edges deleted, as many added); undirected, unlabelled."""
    return [config4_pair(i, nmin, nmax, cid) for i in range(count)]


def config4_train_pair(i: int) -> Pair:
    """Training pair i for the branching network (n <= 30, config id 40)."""
    return config4_pair(i, 16, 30, cid=40)


def config4_train_pairs(count: int = 20000, nmin: int = 16, nmax: int = 30) -> List[Pair]:
    """Training pairs for the branching network: same families as config 4
    with n <= 30 and seeds disjoint from the evaluation pairs (config id 40)."""
    return config4_pairs(count, nmin, nmax, cid=40)


def planted_pair(n: int, core_frac: float, p: float, rng: np.random.Generator) -> Pair:
    """Two G(n, p) graphs sharing a planted induced core of round(core_frac*n)
    vertices (mirrors how ARG ``mcsXX`` pairs are built); H is then permuted."""
    k = int(round(core_frac * n))
    core = er_undirected(k, p, rng)
    G = er_undirected(n, p, rng)
    H = er_undirected(n, p, rng)
    G[:k, :k] = core
    H[:k, :k] = core
    H, _ = _permute(H, None, rng)
    return Pair(Graph(G), Graph(H), False, f"planted-{n}-{k}")


@dataclass
class Request:
    arrival_s: float
    pair: Pair
    timeout_s: float


def config5_requests(count: int = 100000, rate_per_s: float = 1000.0,
                     nmin: int = 16, nmax: int = 56, pmin: float = 0.05,
                     pmax: float = 0.4, kmax: int = 8, timeout_s: float = 1.0,
                     cid: int = 5) -> Iterator[Request]:
    """Poisson arrival stream: exponential gaps at ``rate_per_s``; n
    log-uniform in [nmin, nmax]; p U[pmin, pmax]; k ~ U{0..kmax} label
    classes shared by both graphs of a request (k == 0: unlabelled)."""
    t = 0.0
    arr = np.random.Generator(np.random.PCG64(np.random.SeedSequence([cid, 1 << 30, 0])))
    for i in range(count):
        t += float(arr.exponential(1.0 / rate_per_s))
        r0 = rng_for(cid, i, 0)
        k = int(r0.integers(0, kmax + 1))
        gs = []
        for side in (0, 1):
            r = rng_for(cid, i, side + 1)
            n = int(round(np.exp(r.uniform(np.log(nmin), np.log(nmax)))))
            p = float(r.uniform(pmin, pmax))
            gs.append(Graph(er_undirected(n, p, r), uniform_labels(n, k, r)))
        yield Request(t, Pair(gs[0], gs[1], False, f"c5-{i}"), timeout_s)

def planted_bvg_pair(i: int, nmin: int = 40, nmax: int = 64, cid: int = 44) -> Pair:
    """Bounded-valence pair with a planted common induced core, the way the
    ARG ``mcs10``..``mcs90`` pairs are built: a core of round(f * n) vertices,
    f in {0.1, 0.3, 0.5, 0.7, 0.9} by i, is a random 3-regular graph (even i)
    or a 2D mesh (odd i); each graph adds its own n - k vertices, each joined
    to two or three random vertices; H is then randomly permuted.  The common
    core makes the MCS at least k."""
    r = rng_for(cid, i, 0)
    n = int(r.integers(nmin, nmax + 1))
    f = (0.1, 0.3, 0.5, 0.7, 0.9)[i % 5]
    k = max(4, int(round(f * n)))
    if i % 2 == 0:
        if (k * 3) % 2:
            k -= 1
        core = random_regular(k, 3, r)
    else:
        w = max(2, int(round(np.sqrt(k))))
        h = max(2, k // w)
        k = w * h
        core = grid(w, h)
    gs = []
    for side in (0, 1):
        rs = rng_for(cid, i, side + 1)
        a = np.zeros((n, n), np.uint8)
        a[:k, :k] = core
        for x in range(k, n):
            deg = int(rs.integers(2, 4))
            for y in rs.choice(x, size=min(deg, x), replace=False):
                a[x, y] = a[y, x] = 1
        gs.append(a)
    perm = rng_for(cid, i, 3).permutation(n)
    return Pair(Graph(gs[0]), Graph(gs[1][np.ix_(perm, perm)]), False, f"pbvg-{cid}-{i}")
