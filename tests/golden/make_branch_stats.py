"""Training data for the branching-order network, from the CPU oracle.

Calls only ``oracle/`` (and the seeded generators in ``synth/``).  For each
training pair (bounded-valence family, n <= 30, seeds disjoint from the
evaluation pairs) the oracle's instrumented McSplit logs every branching
decision at depth <= MAX_DEPTH: the chosen G vertex v and each candidate u.
A candidate is a positive example when the search below (v, u) raised the
incumbent to the final optimum, else a negative one.  Pairs whose search did
not finish within the node limit are skipped (their optimum is unknown).
All positives are kept; negatives are subsampled (seeded) to at most NEG
per positive of the same pair.

    python tests/golden/make_branch_stats.py --count 20000 --workers 6

Output: ``tests/golden/order_train.npz`` with int32 columns pair, v, u
(original vertex ids) and uint8 y.
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

MAX_DEPTH = 2          # log decisions at depth 0 and 1
NODE_LIMIT = 300000
NEG = 4


FAMILY = "bvg"


def _one(args):
    i, family, node_limit = args
    import oracle
    import synth
    p = _pair(i) if family == "bvg" else synth.planted_bvg_pair(i, 16, 30, cid=46)
    rows, pg, ph, size, complete = oracle.branch_log(p.G.adj, p.H.adj, max_depth=MAX_DEPTH,
                                                     node_limit=node_limit)
    if not complete or len(rows) == 0:
        return i, None
    v = pg[rows[:, 1]]
    u = ph[rows[:, 2]]
    y = (rows[:, 4] == size).astype(np.uint8)
    pos = np.nonzero(y == 1)[0]
    neg = np.nonzero(y == 0)[0]
    r = np.random.default_rng(1000003 * i + 7)
    keep_neg = neg if len(neg) <= NEG * max(1, len(pos)) else r.choice(neg, NEG * max(1, len(pos)), replace=False)
    keep = np.sort(np.concatenate([pos, keep_neg]))
    return i, (v[keep].astype(np.int32), u[keep].astype(np.int32), y[keep])


def _pair(i):
    # config4_train_pairs draws pair i from its own seed; build it directly
    import synth
    fam = i % 2
    gs = [synth._c4_graph(synth.rng_for(40, i, s), 16, 30, fam) for s in (0, 1)]
    return synth.Pair(synth.Graph(gs[0]), synth.Graph(gs[1]), False, f"c4t-{i}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=20000)
    ap.add_argument("--workers", type=int, default=6)
    ap.add_argument("--family", default="bvg", choices=["bvg", "planted"],
                    help="bvg: random 3-/4-regular and perturbed meshes; planted: "
                         "bounded-valence pairs with a planted common core (synth.planted_bvg_pair)")
    ap.add_argument("--node-limit", type=int, default=NODE_LIMIT)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    out_path = a.out or os.path.join(HERE, "order_train.npz" if a.family == "bvg" else "order_train_planted.npz")
    ctx = mp.get_context("spawn")
    cols = {"pair": [], "v": [], "u": [], "y": []}
    done = 0
    with ctx.Pool(a.workers) as pool:
        for i, res in pool.imap_unordered(_one, [(i, a.family, a.node_limit) for i in range(a.count)], chunksize=16):
            done += 1
            if res is not None:
                v, u, y = res
                cols["pair"].append(np.full(len(v), i, np.int32))
                cols["v"].append(v)
                cols["u"].append(u)
                cols["y"].append(y)
            if done % 1000 == 0:
                print(done, flush=True)
    out = {k: np.concatenate(c) for k, c in cols.items()}
    order = np.lexsort((out["u"], out["v"], out["pair"]))
    out = {k: c[order] for k, c in out.items()}
    np.savez_compressed(out_path, count=np.int32(a.count), max_depth=np.int32(MAX_DEPTH),
                        node_limit=np.int64(a.node_limit), family=a.family, **out)
    print("rows", len(out["y"]), "positives", int(out["y"].sum()),
          "pairs", len(np.unique(out["pair"])))


if __name__ == "__main__":
    main()
