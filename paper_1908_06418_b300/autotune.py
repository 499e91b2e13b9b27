"""Autotuner for the search kernel's launch shape.

    python -m paper_1908_06418_b300.autotune --workload c3 --workload c2

For each workload it times device-resident batch solves (inputs already in
HBM, CUDA events on the launching stream, best of `--reps`) over a grid of
launch shapes -- lanes per searcher (32: one search per warp; 16, 8, 4, 2:
two to sixteen per warp), warps per block, class-stack entries kept in shared
memory per whole-warp searcher (which sets shared memory per warp and so the
resident warps), and blocks per SM -- then, on the fastest shape, the
work-sharing poll interval and the share a donor keeps, and records the
fastest setting for the workload's bucket
(directed or not, labelled or not, largest vertex count rounded up to 32 /
48 / 64) in ``data/tune_cache.json``.  ``Solver.apply_tuned(pairs)`` applies
the cached shape for a batch's bucket.

Buckets whose pairs run into the per-pair limit (the bounded-valence batch:
no pair is proven within a second) are ranked by search nodes per second
over a fixed limit instead of by time to solve (``objective="nodes"``).
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "data", "tune_cache.json")

SHAPES = ([dict(search_group=32, warps_per_block=w, smem_stack_entries=s, blocks_per_sm=0)
           for w, s in itertools.product((4,), (128, 256))]
          # narrow searchers keep class stacks in global memory: no shared-memory size to sweep
          + [dict(search_group=g, warps_per_block=w, smem_stack_entries=-1, blocks_per_sm=0)
             for g, w in ((16, 4), (8, 2), (8, 4), (8, 8), (4, 2), (4, 4), (4, 8), (2, 4))])
KEYS = ("search_group", "warps_per_block", "smem_stack_entries", "blocks_per_sm")
# second stage, on the fastest shape: work-sharing poll interval x the donor's kept share
STEAL = [dict(poll_nodes=pn, steal_keep_quarters=kq) for pn, kq in itertools.product((8, 16, 32), (1, 2, 3))]


def bucket(pairs, directed: bool) -> str:
    nmax = max(max(p.G.n, p.H.n) for p in pairs)
    nb = 32 if nmax <= 32 else (48 if nmax <= 48 else 64)
    lab = any(p.G.labels is not None for p in pairs)
    return f"{'dir' if directed else 'und'}-{'lab' if lab else 'unl'}-n{nb}"


def load_cache(path: str = CACHE) -> dict:
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def time_shape(solver, batch, n, shape, reps, timeout_s):
    import torch
    from . import MCS_OK
    dev = batch.device
    out = dict(size=torch.zeros(n, dtype=torch.int32, device=dev),
               status=torch.zeros(n, dtype=torch.int32, device=dev),
               nodes=torch.zeros(n, dtype=torch.int64, device=dev))
    solver.set_launch(shape["warps_per_block"], shape["blocks_per_sm"] or -1, shape["smem_stack_entries"],
                      search_group=shape["search_group"])
    solver.set_steal(shape.get("poll_nodes", -1), shape.get("steal_keep_quarters", -1))
    stream = torch.cuda.Stream(dev)
    best = None
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = solver.solve_batch_device(n, batch.d_n, batch.d_adj_off, batch.d_adj, batch.d_lab_off,
                                       batch.d_labels, out["size"], out["status"], out["nodes"],
                                       flags=batch.flags, timeout_s=timeout_s,
                                       stream=stream.cuda_stream)
        e1.record(stream)
        stream.synchronize()
        if rc != 0 or not bool((out["status"] == MCS_OK).all()):
            return None
        if r > 0:
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
    return best


def rate_shape(solver, batch, n, shape, reps, timeout_s):
    """Best search-node rate (nodes per microsecond of kernel time) of the
    shape over `reps` device solves that stop at the per-pair limit; None if
    a call fails."""
    import torch
    dev = batch.device
    out = dict(size=torch.zeros(n, dtype=torch.int32, device=dev),
               status=torch.zeros(n, dtype=torch.int32, device=dev),
               nodes=torch.zeros(n, dtype=torch.int64, device=dev))
    solver.set_launch(shape["warps_per_block"], shape["blocks_per_sm"] or -1, shape["smem_stack_entries"],
                      search_group=shape["search_group"])
    solver.set_steal(shape.get("poll_nodes", -1), shape.get("steal_keep_quarters", -1))
    stream = torch.cuda.Stream(dev)
    best = None
    for r in range(reps + 1):
        rc = solver.solve_batch_device(n, batch.d_n, batch.d_adj_off, batch.d_adj, batch.d_lab_off,
                                       batch.d_labels, out["size"], out["status"], out["nodes"],
                                       flags=batch.flags, timeout_s=timeout_s, stream=stream.cuda_stream)
        stream.synchronize()
        if rc < 0:
            return None
        st = solver.last_stats()
        if r > 0 and st["kernel_us"] > 0:
            rate = int(out["nodes"].sum().item()) / st["kernel_us"]
            best = rate if best is None else max(best, rate)
    return best


def tune(name: str, pairs, directed: bool, reps: int = 2, timeout_s: float = 120.0,
         cache_path: str = CACHE, objective: str = "time") -> dict:
    """objective "time": fastest batch solve (ms); "nodes": highest search-node
    rate over solves cut at `timeout_s` per pair (nodes per microsecond)."""
    from . import Solver, DeviceBatch
    batch = DeviceBatch(pairs, directed=directed)
    measure = time_shape if objective == "time" else rate_shape
    field = "ms" if objective == "time" else "nodes_per_us"
    pick = min if objective == "time" else max
    results = []
    with Solver(0) as s:
        for shape in SHAPES:
            t = measure(s, batch, len(pairs), shape, reps, timeout_s)
            results.append(dict(shape, **{field: t}))
            print(name, shape, t, flush=True)
        ok = [r for r in results if r[field] is not None]
        best = {k: pick(ok, key=lambda r: r[field])[k] for k in KEYS}
        steal = []
        for st in STEAL:
            shape = dict(best, **st)
            t = measure(s, batch, len(pairs), shape, reps, timeout_s)
            steal.append(dict(shape, **{field: t}))
            print(name, shape, t, flush=True)
    ok = [r for r in steal if r[field] is not None]
    best = pick(ok, key=lambda r: r[field])
    cache = load_cache(cache_path)
    key = bucket(pairs, directed)
    cache[key] = dict(best, workload=name, measured=time.strftime("%Y-%m-%d"),
                      sweep=[{k: r[k] for k in KEYS + (field,)} for r in results],
                      steal_sweep=[{k: r[k] for k in ("poll_nodes", "steal_keep_quarters", field)} for r in steal])
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    with open(cache_path, "w") as f:
        json.dump(cache, f, indent=1)
    return cache[key]


def main():
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", action="append", default=[])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--cache", default=CACHE)
    a = ap.parse_args()
    for w in a.workload or ["c3"]:
        if w == "c2":
            ps = [p for p in synth.config2_pairs() if p.directed]
            tune(w, ps, True, a.reps, cache_path=a.cache)
        elif w == "c2u":
            ps = [p for p in synth.config2_pairs() if not p.directed]
            tune(w, ps, False, a.reps, cache_path=a.cache)
        elif w == "c3":
            tune(w, synth.config3_pairs(), False, a.reps, cache_path=a.cache)
        elif w == "c1":
            tune(w, synth.config1_like(64), False, a.reps, cache_path=a.cache)
        elif w == "c4":
            # no pair is proven within the limit: rank shapes by node rate over 0.3 s per pair
            tune(w, synth.config4_pairs(2048), False, a.reps, timeout_s=0.3, cache_path=a.cache,
                 objective="nodes")
        else:
            raise SystemExit(f"unknown workload {w}")


if __name__ == "__main__":
    main()
