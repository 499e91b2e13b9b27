"""Writes stored oracle results for the synthetic workloads.

Calls only ``oracle/`` (and the seeded generators in ``synth/``).  Every stored
size comes from the CPU oracle; nothing here touches the CUDA path.

    python tests/golden/make_oracle_golden.py c2 --budget 1800 --workers 5
    python tests/golden/make_oracle_golden.py c3 --budget 10 --workers 6
    python tests/golden/make_oracle_golden.py c4 --budget 10 --count 256
    python tests/golden/make_oracle_golden.py c5 --budget 60 --count 800
    python tests/golden/make_oracle_golden.py c4p --budget 300 --workers 3
    python tests/golden/make_oracle_golden.py planted --budget 300 --workers 2

Output: ``tests/golden/<cfg>_oracle.jsonl``, one JSON object per pair with the
pair index, a digest of both adjacency matrices (to detect generator drift),
the size, whether the search completed within the budget (size proven
optimal), the node count, seconds and the mapping in original vertex ids.

``c4p`` is the planted-core form of the bounded-valence workload: 96 pairs of
40 to 64 vertices whose graphs share a common induced core of 90 % of n (the
way the ARG ``mcsXX`` pairs are built).  Unrelated bounded-valence pairs of
that size are beyond the oracle's reach, so these give the workload an exact
check.  They are solved with the oracle's top-down strategy (Section IV-A),
which is exact and finishes fastest when the optimum is near min(n_G, n_H).

``planted`` is the held-out planted-core family the ordering network is
measured on: 160 bounded-valence pairs of 24 to 34 vertices with cores of 10
to 90 % of n, solved with the plain oracle.
"""
from __future__ import annotations

import argparse
import hashlib
import itertools
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def pair_digest(p) -> str:
    h = hashlib.sha1()
    for g in (p.G, p.H):
        h.update(g.adj.tobytes())
        if g.labels is not None:
            h.update(g.labels.tobytes())
    h.update(b"d" if p.directed else b"u")
    return h.hexdigest()[:16]


def load_pairs(cfg: str, count: int):
    import synth
    if cfg == "c1":
        return [synth.config1_pair()]
    if cfg == "c1x":
        return synth.config1_like(count or 64)
    if cfg == "c2":
        return synth.config2_pairs()
    if cfg == "c3":
        return synth.config3_pairs(count=count or 4096)
    if cfg == "c4":
        return synth.config4_pairs(count=count or 2048)
    if cfg == "c4p":
        return c4p_pairs()
    if cfg == "planted":
        import synth
        return [synth.planted_bvg_pair(i, 24, 34, cid=47) for i in range(count or 160)]
    if cfg == "c5":
        return [r.pair for r in itertools.islice(synth.config5_requests(count=count or 2000),
                                                  count or 2000)]
    raise ValueError(cfg)


def c4p_pairs():
    """Planted-core bounded-valence pairs, 40 to 64 vertices, core 90 % of n."""
    import synth
    return [synth.planted_bvg_pair(i, 40, 64, cid=62) for i in range(4, 480, 5)]


def _work(args):
    cfg, idx, count, budget = args
    import oracle
    p = load_pairs(cfg, count)[idx] if cfg in ("c1", "c2") else _cached(cfg, count)[idx]
    t = time.time()
    run = oracle.mcs_topdown if cfg == "c4p" else oracle.mcs
    r = run(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=p.directed, time_limit_s=budget)
    dt = time.time() - t
    return dict(idx=idx, tag=p.tag, nG=p.G.n, nH=p.H.n, directed=p.directed,
                digest=pair_digest(p), size=r.size, complete=bool(r.complete),
                nodes=r.nodes, seconds=round(dt, 4),
                g=[int(x) for x in r.g_idx], h=[int(x) for x in r.h_idx])


_CACHE = {}


def _cached(cfg, count):
    key = (cfg, count)
    if key not in _CACHE:
        _CACHE[key] = load_pairs(cfg, count)
    return _CACHE[key]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cfg")
    ap.add_argument("--budget", type=float, default=10.0)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--count", type=int, default=0)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    n = len(load_pairs(a.cfg, a.count))
    out = a.out or os.path.join(HERE, f"{a.cfg}_oracle.jsonl")
    done = {}
    if os.path.exists(out):
        for line in open(out):
            if line.strip():
                d = json.loads(line)
                done[d["idx"]] = d
    todo = [(a.cfg, i, a.count, a.budget) for i in range(n) if i not in done]
    # hardest-looking first is not knowable in advance; keep index order
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.workers) as pool, open(out, "a") as f:
        for d in pool.imap_unordered(_work, todo):
            f.write(json.dumps(d) + "\n")
            f.flush()
            print(d["idx"], d["tag"], d["size"], d["complete"], d["seconds"], flush=True)
    # rewrite sorted by index
    rows = {}
    for line in open(out):
        if line.strip():
            d = json.loads(line)
            rows[d["idx"]] = d
    with open(out, "w") as f:
        for i in sorted(rows):
            f.write(json.dumps(rows[i]) + "\n")


if __name__ == "__main__":
    main()
