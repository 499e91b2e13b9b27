"""Benchmark: exact MCS pairs solved/sec and search nodes/sec on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2|c3|c1|c4|c5|td]
                    [--impl ours|reference]

A step solves one whole workload batch: every pair of the workload, each to a
proven optimum (status MCS_OK).  Default workload: the hard single pairs --
96 directed unlabelled G(36, p) pairs, p in {0.05, 0.1, 0.3} x 32 seeds, plus
one pair of 6x6 grids with 10% of their edges deleted -- solved as two
persistent launches (one directed, one undirected) with all inputs resident in
HBM.  Timing: CUDA events on the launching stream around each step; the L2
cache (126 MB) is flushed by writing a 512 MB buffer between steps, outside
the timed events.  `value` = pairs solved / summed step time.

Other workloads: c3 (4,096 labelled pairs), c1 (one small pair), c4 (2,048
bounded-valence pairs, learned order, 1 s per pair), c5 (serving on a Poisson
stream), td (96 bounded-valence pairs with a 90 % planted core, solved with
the top-down strategy of Section IV-A; the line adds the plain search, the
dead-end forecast and randomized restarts on the same batch).

`--impl reference` times the CPU oracle (plain sequential McSplit) on the
host cores on a bounded sample of the same workload; it is the reference arm
(there is no reference implementation to install for this paper).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
MCS_MAX_N = 256          # include/mcs.h: stride of the device mapping outputs

METRIC = "MCS pairs solved/sec (exact) on 1 B300"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant search kernel, from a single-pass ncu capture of this
# workload's launch:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none
#       -k regex:search_kernel -s <search launches before the timed one> -c 1
#       python bench.py --workload <w> --steps 2 --warmup 1 --no-cpu-baseline --no-single
#       --no-batched --no-served --no-race
# Reported only while the kernel source is the one the capture was taken with.
TRAFFIC = {"c2": {"kernel_sha1": "bfc9a84d6fb9f8a0", "bytes": 992815360 + 979917568},
           "c3": {"kernel_sha1": "bfc9a84d6fb9f8a0", "bytes": 102537728 + 191992576}}
UNIT = "pairs/s"


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def workload(name: str, shard: int = 0):
    """The named workload's pairs and config.  Under several ranks each rank
    solves shard `shard` = its rank: the same recipe (sizes, densities,
    labels) drawn from seeds of its own, so no pair is solved twice."""
    import synth
    sc = lambda cid: synth.shard_cid(cid, shard)
    if name == "c2":
        return synth.config2_pairs(cid=sc(2)), dict(
            workload="hard single pairs: 96 directed G(36,p), p in {0.05,0.1,0.3} x 32 seeds "
                     "+ 6x6 grid pair with 10% edges deleted", pairs=97)
    if name == "c2s":     # small case of the same kernel for profiler captures
        return synth.config2_pairs(cid=sc(2))[0:96:4], dict(
            workload="24 directed G(36,p) pairs (every 4th of the hard single pairs)", pairs=24)
    if name == "c3":
        return synth.config3_pairs(cid=sc(3)), dict(
            workload="batched: 4096 undirected pairs, n U{10..40}, p U[0.05,0.4], 4 labels",
            pairs=4096)
    if name == "c1":
        return [synth.config1_pair()], dict(workload="single pair G(20,0.3) x G(20,0.3)", pairs=1)
    if name == "c4":
        return synth.config4_pairs(2048, cid=sc(4)), dict(
            workload="learned ordering: 2048 bounded-valence pairs (random 3-/4-regular and perturbed "
                     "2D meshes, n U{40..64}), order network data/order_mlp_bvg.npy (per-pair limit: timeout_s)",
            pairs=2048)
    if name == "td":
        return [synth.planted_bvg_pair(i, 40, 64, cid=sc(62)) for i in range(4, 480, 5)], dict(
            workload="top-down strategy (Section IV-A): 96 bounded-valence pairs with a planted common "
                     "core of 90% of n (3-regular or mesh core), n U{40..64}; MCS_TOP_DOWN", pairs=96)
    raise SystemExit(f"unknown workload {name}")


def golden_sizes(name: str):
    """Stored oracle sizes by position in the workload (c2s: every 4th c2 pair)."""
    stride = 1
    if name == "c2s":
        name, stride = "c2", 4
    path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle.jsonl")
    if not os.path.exists(path):
        return {}
    out = {}
    for line in open(path):
        if line.strip():
            d = json.loads(line)
            if stride == 1:
                out[d["idx"]] = (d["size"], d["complete"])
            elif d["idx"] % stride == 0 and d["idx"] < 96:        # the directed pairs
                out[d["idx"] // stride] = (d["size"], d["complete"])
    return out


# ---------------------------------------------------------------------------
# clocks sampler
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.stop = threading.Event()
        self.th = None

    def _run(self):
        while not self.stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self.stop.wait(0.2)

    def __enter__(self):
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        if self.th:
            self.th.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# CPU oracle (reported baseline / reference arm)
# ---------------------------------------------------------------------------
def _oracle_one(args):
    name, idx, budget = args
    import oracle
    pairs, _ = workload(name)
    p = pairs[idx]
    t = time.time()
    run = oracle.mcs_topdown if name == "td" else oracle.mcs
    r = run(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=p.directed, time_limit_s=budget)
    return idx, r.size, r.complete, r.nodes, time.time() - t


def host_cpu():
    """(usable host cores, CPU model) of this machine."""
    cores = len(os.sched_getaffinity(0))
    model = "unknown"
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return cores, model


def oracle_sample(name: str, n_pairs: int, budget: float, offset: int = 0):
    """Runs the oracle over a bounded sample (every k-th pair) with one worker
    process per usable host core; the sample has at least one pair per core
    (up to the workload's size), so every core works."""
    pairs, _ = workload(name)
    cores, model = host_cpu()
    n_pairs = min(len(pairs), max(n_pairs, cores))
    step = max(1, len(pairs) // n_pairs)
    idx = [(offset + i * step) % len(pairs) for i in range(n_pairs)]
    gold = golden_sizes(name)
    ctx = mp.get_context("spawn")
    t = time.time()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_one, [(name, i, budget) for i in idx], chunksize=1)
    wall = time.time() - t
    solved = sum(1 for (i, k, c, n, s) in res if c and (i not in gold or gold[i][0] == k or not gold[i][1]))
    nodes = sum(n for (_, _, _, n, _) in res)
    lat = sorted(s for (_, _, c, _, s) in res if c)
    return dict(solved=solved, tried=len(idx), wall=wall, nodes=nodes, cores=cores, cpu_model=model,
                p99=(float(np.percentile(lat, 99)) if lat else None),
                sample=f"{len(idx)} of {len(pairs)} pairs (every {step}th), {budget:g} s budget per pair, "
                       f"one worker process per host core ({cores} cores, {model})")


def combine_ranks(total_ms, solved, nodes, dist=None, device="cpu"):
    """Whole-job figures of a multi-rank run (one shard of pairs per rank): after a
    barrier, the slowest rank's timed milliseconds and the work of all ranks
    summed.  dist: torch.distributed (any backend) or None for one rank."""
    if not dist:
        return total_ms, solved, nodes
    import torch
    dist.barrier()
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([solved, nodes], dtype=torch.float64, device=device)
    dist.all_reduce(w)
    return float(t.item()), int(w[0].item()), int(w[1].item())


def apply_shape(solver, sh):
    """The autotuned launch shape of a group, else the library's defaults."""
    if sh:
        solver.set_launch(sh["warps_per_block"], sh["blocks_per_sm"] or -1, sh["smem_stack_entries"],
                          search_group=sh["search_group"])
        solver.set_steal(sh["poll_nodes"], sh["steal_keep_quarters"])
    else:
        solver.reset_launch()


def single_instance_vs_batch(solver, pairs, a, batch_flags=0):
    """The plain single-instance form on the same GPU: a bounded sample of the
    workload solved one pair per mcs_solve call (whole-warp searchers, the
    tuned shape for single pairs, degree order), in FIFO order from t = 0,
    against the same sample as one mcs_solve_batch call with the workload's
    tuned shape (and batch_flags, e.g. the learned order).
    Both go through the host C ABI (copies included).  Latency of a pair =
    time from t = 0 to its result."""
    import torch
    from paper_1908_06418_b300 import MCS_OK, MCS_DIRECTED, HostBatch
    n = len(pairs)
    k = {"c2": 24, "c2s": 8, "c3": 256, "c1": 1, "c4": 8, "td": 8}.get(a.workload, min(n, 64))
    idx = list(range(0, n, max(1, n // k)))[:k]
    sample = [pairs[i] for i in idx]
    # one pair per call
    solver.set_launch(4, -1, 256, search_group=32)
    solver.set_steal(-1, -1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done, ok1 = [], 0
    for p in sample:
        r = solver.solve(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=bool(p.directed),
                         timeout_s=a.timeout)
        done.append((time.perf_counter() - t0) * 1e3)
        ok1 += int(r.status == MCS_OK)
    t_single = done[-1] / 1e3
    # the same sample as one batch per flag group
    t0 = time.perf_counter()
    ok2 = 0
    for directed in (True, False):
        sub = [p for p in sample if bool(p.directed) == directed]
        if not sub:
            continue
        solver.apply_tuned(sub, directed=directed) or solver.reset_launch()
        out = solver.solve_host(HostBatch(sub, directed=directed), flags=batch_flags, timeout_s=a.timeout)
        ok2 += int((out["status"] == MCS_OK).sum())
    t_batch = time.perf_counter() - t0
    solver.reset_launch()
    return {"sample": f"{len(sample)} of {n} pairs (every {max(1, n // k)}th)",
            "single_pairs_s": ok1 / t_single, "single_p50_ms": float(np.percentile(done, 50)),
            "single_p99_ms": float(np.percentile(done, 99)),
            "batch_pairs_s": ok2 / t_batch, "batch_p99_ms": t_batch * 1e3,
            "note": "latency from t = 0: FIFO one pair per call vs all pairs in one batch call"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = a.workload
    n_sample = 8 if name.startswith("c2") else 64
    budget = a.timeout if name == "c4" else (25.0 if name.startswith("c2") else 2.0)
    for w in range(a.warmup):
        oracle_sample(name, 2, 0.5, offset=w)
    tot_solved = tot_wall = tot_nodes = 0
    last = None
    for k in range(a.steps):
        r = oracle_sample(name, n_sample, budget, offset=k)
        tot_solved += r["solved"]
        tot_wall += r["wall"]
        tot_nodes += r["nodes"]
        last = r
    val = tot_solved / tot_wall if tot_wall else 0.0
    _, cfg = workload(name)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * tot_wall / max(1, a.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "nodes_per_s": tot_nodes / tot_wall if tot_wall else 0.0,
            "config": dict(cfg, sample=last["sample"]),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "cpu_model": last["cpu_model"], "sample": last["sample"]},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--order", default="degree", choices=["degree", "hr"],
                    help="vertex order of the search: degree (default) or the static component + "
                         "Hellerman-Rarick-style order of Section IV-A (MCS_ORDER_HR; not with c4's learned order)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--timeout", type=float, default=None,
                    help="per-pair limit in seconds (default 600; c4: 1)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="ignore the autotuner cache")
    ap.add_argument("--no-single", action="store_true",
                    help="skip the single-instance (one pair per call) comparison")
    ap.add_argument("--no-batched", action="store_true",
                    help="default run: skip the batched (c3) key")
    ap.add_argument("--no-served", action="store_true",
                    help="default run: skip the served (c5) key")
    ap.add_argument("--no-race", action="store_true",
                    help="default run: skip the GPU + CPU race sample (race key)")
    ap.add_argument("--requests", type=int, default=100000, help="c5: requests in the stream")
    ap.add_argument("--rate-frac", type=float, default=0.5, help="c5: arrival rate / saturated rate")
    ap.add_argument("--rate", type=float, default=0.0, help="c5: absolute arrival rate (requests/s), "
                                                             "instead of --rate-frac")
    ap.add_argument("--single-sample", type=int, default=300, help="c5: single-instance baseline sample")
    ap.add_argument("--serve-lanes", type=int, default=0,
                    help="c5: lanes per searcher of the server (8, 16 or 32; default: the library's, 32)")
    a = ap.parse_args(argv)
    if a.timeout is None:
        a.timeout = 1.0 if a.workload == "c4" else 600.0
    return a


def main():
    a = parse_args()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.workload == "c5":
        print(json.dumps(run_serving(a)), flush=True)
        return

    import copy
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1908_06418_b300 import Solver
    solver = Solver(local)
    line = measure(a, a.workload, solver, local, rank, world, dist)
    # the default run (one GPU) also measures the batched form (the 4,096
    # labelled pairs) and the served form (the Poisson stream of requests);
    # under several ranks only the sharded headline workload runs
    if world == 1 and a.workload == "c2" and not a.no_batched:
        b = copy.copy(a)
        b.workload = "c3"
        sub = measure(b, "c3", solver, local, rank, world, None)
        line["batched"] = {k: sub[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "warmup",
                                                "nodes_per_s", "p50_latency_ms", "p99_latency_ms",
                                                "solved_per_step", "config", "gpu_launches", "e2e",
                                                "roofline", "clocks", "single_instance", "cpu_baseline")
                           if k in sub}
    if world == 1 and a.workload == "c2" and not a.no_race:
        line["race"] = race_sample(solver, a)
    solver.close()
    if world == 1 and a.workload == "c2" and not a.no_served:
        line["served"] = run_serving(a)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def measure(a, name, solver, local, rank, world, dist):
    """One workload on the device: K timed steps after W warm-up steps (each
    step solves every pair of the workload), then the same workload end to end
    through the host C ABI, the roofline of the dominant kernel, and the
    comparisons.  Returns the bench line (dict)."""
    import torch
    from paper_1908_06418_b300 import (pack_host, MCS_DIRECTED, MCS_OK, MCS_WORD32, MCS_ORDER_LEARNED,
                                       MCS_TOP_DOWN, MCS_DEAD_END, MCS_ORDER_HR, MCS_RESTART)

    # each rank its own shard of pairs; the stored oracle sizes cover shard 0
    pairs, cfg = workload(name, shard=rank)
    gold = golden_sizes(name) if rank == 0 else {}
    dev = torch.device("cuda", local)
    learned = name == "c4" and a.order == "degree"
    hr = a.order == "hr"
    topdown = name == "td"
    if learned:       # the candidate order of the trained network (exactness unchanged)
        solver.set_order_model(np.load(os.path.join(ROOT, "paper_1908_06418_b300", "data",
                                                    "order_mlp_bvg.npy")).astype(np.float32))
    # a dedicated stream: the library's device entry point runs on the stream
    # it is given, and CUDA events recorded on that same stream time it
    stream = torch.cuda.Stream(dev)

    # device-resident inputs, one group per flag set (this rank's shard);
    # a group whose graphs all have at most 32 vertices takes the 32-bit node step
    groups = []
    for directed in (True, False):
        idx = [i for i, p in enumerate(pairs) if p.directed == directed]
        if not idx:
            continue
        narrow = all(max(pairs[i].G.n, pairs[i].H.n) <= 32 for i in idx)
        h = pack_host([pairs[i] for i in idx])
        g = dict(idx=idx, flags=(MCS_DIRECTED if directed else 0) | (MCS_WORD32 if narrow else 0)
                 | (MCS_ORDER_LEARNED if learned else 0) | (MCS_TOP_DOWN if topdown else 0)
                 | (MCS_ORDER_HR if hr else 0), n=len(idx),
                 d_n=torch.from_numpy(h["n"]).to(dev),
                 d_adj_off=torch.from_numpy(h["adj_off"]).to(dev),
                 d_adj=torch.from_numpy(h["adj"]).to(dev),
                 d_lab_off=torch.from_numpy(h["lab_off"]).to(dev),
                 d_labels=(torch.from_numpy(h["labels"]).to(dev) if h["labels"] is not None else None),
                 size=torch.zeros(len(idx), dtype=torch.int32, device=dev),
                 status=torch.zeros(len(idx), dtype=torch.int32, device=dev),
                 nodes=torch.zeros(len(idx), dtype=torch.int64, device=dev),
                 usec=torch.zeros(len(idx), dtype=torch.float32, device=dev),
                 map=torch.zeros(len(idx) * MCS_MAX_N, dtype=torch.int16, device=dev))
        groups.append(g)
    # launch shapes recorded by the autotuner for each group's bucket
    shapes = []
    for g in groups:
        e = None if a.no_tune else solver.apply_tuned([pairs[i] for i in g["idx"]],
                                                      directed=bool(g["flags"] & MCS_DIRECTED))
        shapes.append(None if e is None else dict({k: e[k] for k in ("warps_per_block", "smem_stack_entries",
                                                                      "blocks_per_sm")},
                                                  search_group=e.get("search_group", 32),
                                                  poll_nodes=e.get("poll_nodes", -1),
                                                  steal_keep_quarters=e.get("steal_keep_quarters", -1)))
        g["shape"] = shapes[-1]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    launches_per_step = 2 * len(groups)      # pack + search per group

    stats = []   # per timed step: [(group, search_us, class_visits, busy, idle, pruned)]

    def step(evs=None):
        rec = []
        for gi, g in enumerate(groups):
            sh = g.get("shape")
            apply_shape(solver, sh)
            if evs is not None:
                evs[gi][0].record(stream)
            rc = solver.solve_batch_device(g["n"], g["d_n"], g["d_adj_off"], g["d_adj"],
                                           g["d_lab_off"], g["d_labels"], g["size"], g["status"],
                                           g["nodes"], g["map"], g["usec"], flags=g["flags"],
                                           timeout_s=a.timeout, stream=stream.cuda_stream)
            if evs is not None:
                evs[gi][1].record(stream)
                stream.synchronize()
                st = solver.last_stats()
                rec.append((gi, st["kernel_us"], st["class_visits"], st["busy_cycles"],
                            st["idle_cycles"], st["pruned"]))
            if rc != 0:
                raise RuntimeError(f"enqueue failed: {solver.strerror(rc)}")
        if evs is not None:
            stats.append(rec)

    def check():
        solved = 0
        nodes = 0
        lat = []
        for g in groups:
            st = g["status"].cpu().numpy()
            sz = g["size"].cpu().numpy()
            nd = g["nodes"].cpu().numpy()
            us = g["usec"].cpu().numpy()
            for j, i in enumerate(g["idx"]):
                ok = st[j] == MCS_OK
                if ok and i in gold:
                    k, complete = gold[i]
                    ok = (sz[j] == k) if complete else (sz[j] >= k)
                    if not ok:
                        raise SystemExit(f"PARITY FAILURE pair {i}: gpu {sz[j]} oracle {k}")
                solved += int(ok)
                lat.append(us[j] / 1e3)
            nodes += int(nd.sum())
        return solved, nodes, lat

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    flush.fill_(1)

    step_ms, search_ms, solved_tot, nodes_tot, lats = [], [], 0, 0, []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(a.steps):
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in groups]
            step(evs)
            torch.cuda.synchronize()
            step_ms.append(sum(e0.elapsed_time(e1) for e0, e1 in evs))
            search_ms.append(sum(r[1] for r in stats[-1]) / 1e3)
            s, n, l = check()
            solved_tot += s
            nodes_tot += n
            lats += l
            flush.fill_(k & 0xff)          # evict L2 between timed steps (untimed)
            torch.cuda.synchronize()
    total_ms, solved_tot, nodes_tot = combine_ranks(sum(step_ms), solved_tot, nodes_tot, dist, dev)
    value = solved_tot / (total_ms / 1e3)
    nodes_per_s = nodes_tot / (total_ms / 1e3)

    # ---- end to end through the host C ABI: mcs_solve_batch on graphs held in
    # host memory (the library stages them in pinned memory, copies them in,
    # solves and copies the results back inside the timed region)
    from paper_1908_06418_b300 import HostBatch
    hbs = [HostBatch([pairs[i] for i in g["idx"]], directed=bool(g["flags"] & MCS_DIRECTED)) for g in groups]
    e2e_ms, e2e_solved, h2d, d2h = [], 0, 0, 0
    for g, hb in zip(groups, hbs):           # untimed: the bytes each call copies
        apply_shape(solver, g.get("shape"))
        solver.solve_host(hb, flags=g["flags"], timeout_s=a.timeout)
        st = solver.last_stats()
        h2d += st["h2d_bytes"]
        d2h += st["d2h_bytes"]
    for k in range(max(1, min(a.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs = []
        for g, hb in zip(groups, hbs):
            apply_shape(solver, g.get("shape"))
            outs.append(solver.solve_host(hb, flags=g["flags"], timeout_s=a.timeout))
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        for g, res in zip(groups, outs):
            for j, i in enumerate(g["idx"]):
                ok = res["status"][j] == MCS_OK and (i not in gold or (
                    res["size"][j] == gold[i][0] if gold[i][1] else res["size"][j] >= gold[i][0]))
                e2e_solved += int(ok)
    e2e_value = e2e_solved / (sum(e2e_ms) / 1e3)

    # ---- roofline of the dominant kernel (the search kernel of the group
    # that takes longest).  Algorithmic work per label class read by a node
    # expansion: 4 hardware popcounts undirected (|L1|, |R1| as two 64-bit
    # counts), 12 directed (three of the four parts per side); the popcount
    # unit is the bounding pipe, its sustained device rate is measured live
    # by mcs_bench_popc.
    csum = clk.summary()
    popc_peak = solver.bench_popc() / 1e9
    dom = max(range(len(groups)), key=lambda gi: sum(r[gi][1] for r in stats))
    # hardware popcounts per class read: undirected |L1|, |R1|, directed three
    # parts per side; a 64-bit count is two 32-bit ones
    per_class = (12 if groups[dom]["flags"] & MCS_DIRECTED else 4) // (2 if groups[dom]["flags"] & MCS_WORD32 else 1)
    dom_us = [r[dom][1] for r in stats]
    dom_cv = [r[dom][2] for r in stats]
    busy = sum(r[dom][3] for r in stats)
    idle = sum(r[dom][4] for r in stats)
    achieved = (sum(dom_cv) * per_class / 1e9) / (sum(dom_us) * 1e-6)
    import hashlib
    ksha = hashlib.sha1(open(os.path.join(ROOT, "paper_1908_06418_b300", "csrc", "mcs_kernels.cu"),
                             "rb").read()).hexdigest()[:16]
    tr = TRAFFIC.get(name)
    traffic = tr["bytes"] if tr and tr["kernel_sha1"] == ksha else None
    roof = {"bound": "alu", "achieved": achieved, "peak": popc_peak, "unit": "Gpopc/s",
            "frac": achieved / popc_peak, "traffic": traffic,
            "kernel": "search_kernel<%s>" % ("directed" if groups[dom]["flags"] & MCS_DIRECTED else "undirected"),
            "peak_source": "measured: mcs_bench_popc (device-wide sustained 32-bit popc rate)",
            "class_visits_per_launch": sum(dom_cv) / len(dom_cv), "popc_per_class": per_class,
            "launch_ms": sum(dom_us) / len(dom_us) / 1e3,
            "warp_busy_frac": busy / max(1.0, busy + idle),
            "pruned_per_launch": sum(r[dom][5] for r in stats) / len(stats)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "nodes_per_s": nodes_per_s,
            "p50_latency_ms": float(np.percentile(lats, 50)) if lats else None,
            "p99_latency_ms": float(np.percentile(lats, 99)) if lats else None,
            "solved_per_step": solved_tot / a.steps / world,
            "config": dict(cfg, parallelism=f"pair shards x{world} (one shard of distinct pairs per rank, "
                                            "same recipe)", l2="flushed between steps (512 MB write)",
                           vertex_order=("learned" if learned else a.order),
                           timeout_s=a.timeout, launch_shapes=shapes),
            "gpu_launches": launches_per_step * a.steps,
            "search_ms_per_step": sum(search_ms) / len(search_ms),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "roofline": roof, "clocks": csum}
    if rank == 0 and (learned or topdown):
        # the same batch with and without the strategy under test
        def one_pass(flag_clear, flag_set=0):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for g in groups:
                apply_shape(solver, g.get("shape"))
                solver.solve_batch_device(g["n"], g["d_n"], g["d_adj_off"], g["d_adj"], g["d_lab_off"],
                                          g["d_labels"], g["size"], g["status"], g["nodes"], g["map"],
                                          g["usec"], flags=(g["flags"] & ~flag_clear) | flag_set,
                                          timeout_s=a.timeout,
                                          stream=stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            st = np.concatenate([g["status"].cpu().numpy() for g in groups])
            sz = np.concatenate([g["size"].cpu().numpy() for g in groups])
            nd = sum(int(g["nodes"].sum().item()) for g in groups)
            return {"ms": e0.elapsed_time(e1), "solved": int((st == MCS_OK).sum()),
                    "mean_size": float(sz.mean()), "nodes": nd, "_sizes": sz, "_status": st}
        if learned:
            cmp = {"learned": one_pass(0), "plain": one_pass(MCS_ORDER_LEARNED)}
            key = "order_comparison"
        else:
            cmp = {"top_down": one_pass(0), "plain": one_pass(MCS_TOP_DOWN),
                   "dead_end": one_pass(MCS_TOP_DOWN, MCS_DEAD_END),
                   "restart": one_pass(MCS_TOP_DOWN, MCS_RESTART)}
            key = "strategy_comparison"
            # both are exact: where both proved their result the sizes must agree
            for other in ("top_down", "dead_end", "restart"):
                a_, b_ = cmp[other], cmp["plain"]
                both = (a_["_status"] == MCS_OK) & (b_["_status"] == MCS_OK)
                if not np.array_equal(a_["_sizes"][both], b_["_sizes"][both]):
                    raise SystemExit(f"PARITY FAILURE: {other} and plain optima differ")
        for v in cmp.values():
            v.pop("_sizes"); v.pop("_status")
        line[key] = dict(cmp, note="one pass each over the whole batch; exact either way, "
                                   "solved = proven within the per-pair limit")
        if learned:
            line["mlp"] = mlp_roofline(solver, groups, pairs, stream)
    if rank == 0 and not a.no_single:
        line["single_instance"] = single_instance_vs_batch(
            solver, pairs, a, batch_flags=(MCS_ORDER_LEARNED if learned else 0) | (MCS_TOP_DOWN if topdown else 0))
    if rank == 0 and not a.no_cpu_baseline:
        cb = oracle_sample(name, 8 if name.startswith("c2") else 64,
                           a.timeout if name == "c4" else (25.0 if name.startswith("c2") else 2.0))
        line["cpu_baseline"] = {"value": cb["solved"] / cb["wall"], "unit": UNIT, "cores": cb["cores"],
                                "cpu_model": cb["cpu_model"], "kind": "oracle", "sample": cb["sample"],
                                "nodes_per_s": cb["nodes"] / cb["wall"]}
    return line


def race_sample(solver, a, n_req=200):
    """The GPU + CPU race (MCS_RACE) on single pairs: the C1 pair and the
    first n_req requests of the serving stream (n 16..56), each solved by
    mcs_solve with and without the race, in the single-pair launch shape.
    Reports how often each side finished its proof first and the summed
    solve times; sizes must agree where both are proven."""
    import itertools
    import synth
    from paper_1908_06418_b300 import MCS_OK, MCS_RACE
    pairs = [synth.config1_pair()] + [r.pair for r in itertools.islice(synth.config5_requests(count=n_req), n_req)]
    solver.set_launch(4, -1, 256, search_group=32)
    solver.set_steal(-1, -1)
    wins = {0: 0, 1: 0, 2: 0}
    t_plain = t_race = 0.0
    lat_plain, lat_race = [], []
    for p in pairs:
        t0 = time.perf_counter()
        r0 = solver.solve(p.G.adj, p.H.adj, p.G.labels, p.H.labels, timeout_s=1.0)
        t1 = time.perf_counter()
        r1 = solver.solve(p.G.adj, p.H.adj, p.G.labels, p.H.labels, flags=MCS_RACE, timeout_s=1.0)
        t2 = time.perf_counter()
        wins[int(solver.last_stats()["race_winner"])] += 1
        t_plain += t1 - t0
        t_race += t2 - t1
        lat_plain.append((t1 - t0) * 1e3)
        lat_race.append((t2 - t1) * 1e3)
        if r0.status == MCS_OK and r1.status == MCS_OK and r0.size != r1.size:
            raise SystemExit(f"PARITY FAILURE race vs plain: {r1.size} vs {r0.size}")
    solver.reset_launch()
    return {"pairs": len(pairs), "cpu_first": wins[1], "gpu_first": wins[2], "neither_within_1s": wins[0],
            "plain_s": t_plain, "race_s": t_race,
            "plain_p50_ms": float(np.percentile(lat_plain, 50)), "race_p50_ms": float(np.percentile(lat_race, 50)),
            "plain_p99_ms": float(np.percentile(lat_plain, 99)), "race_p99_ms": float(np.percentile(lat_race, 99)),
            "how": "mcs_solve per pair (C1 pair + first serving requests), 1 s limit, with and without MCS_RACE"}


def mlp_roofline(solver, groups, pairs, stream, reps=20):
    """The all-pairs scoring pass of the learned order (vertex features, then
    the tcgen05 MLP forward over every (v, u) of every pair) on the bench's
    batch, timed with CUDA events on its stream.  Algorithmic work counts the
    valid rows only (v < n_G, u < n_H) at 2 x (36 x 128 + 128 x 128 + 128)
    flops each (the unpadded network); the time includes the features kernel,
    so the fraction is a lower bound for the forward kernel alone."""
    import torch
    from types import SimpleNamespace
    peak, src = _tensor_peak()
    outs, views = [], []
    for g in groups:
        views.append(SimpleNamespace(npairs=g["n"], d_n=g["d_n"], d_adj_off=g["d_adj_off"], d_adj=g["d_adj"],
                                     d_lab_off=g["d_lab_off"], d_labels=g["d_labels"], flags=g["flags"],
                                     device=g["d_n"].device))
        outs.append(torch.empty((g["n"], 64, 64), dtype=torch.float32, device=g["d_n"].device))
    for _ in range(3):
        for v, o in zip(views, outs):
            solver.order_score_grid(v, out=o, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        for v, o in zip(views, outs):
            solver.order_score_grid(v, out=o, stream=stream)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / reps
    rows = sum(p.G.n * p.H.n for p in pairs)
    tflops = rows * 2.0 * (36 * 128 + 128 * 128 + 128) / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "kernel": "mlp_fwd_kernel (tcgen05.mma kind::f16, TMEM accumulators)",
            "rows": rows, "ms_per_pass": ms, "rows_per_s": rows / (ms * 1e-3),
            "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
            "peak_source": src,
            "note": "features + forward per pass, inputs resident; fp16 operands, fp32 accumulation"}


def _tensor_peak():
    """Dense fp16 tensor peak: the measured bf16 burst figure (fp16 and bf16
    run at the same nominal dense rate on this part)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "of measured (bf16 burst; fp16 nominal ratio 1)"
    except (OSError, KeyError, ValueError):
        return 1800.0, "of fallback (1.8 PFLOP/s bf16 burst; fp16 nominal ratio 1)"


# ---------------------------------------------------------------------------
# serving (continuous batching) on a Poisson stream
# ---------------------------------------------------------------------------
def run_serving(a):
    """The served form: a Poisson stream of config-5 requests (n log-uniform
    16..56, 0-8 label classes, 1 s limit each) through mcs_submit/mcs_poll,
    at a fraction of the batch solver's saturated rate (or --rate); latency =
    arrival -> result on the host.  Beside it, the plain single-instance form
    (one mcs_solve per request, FIFO at the same arrival times) on a sample.
    Returns the line (dict)."""
    import itertools
    import torch
    import synth
    from paper_1908_06418_b300 import Solver, MCS_OK, MCS_TIMEOUT
    torch.cuda.set_device(0)
    solver = Solver(0)
    n_req = a.requests
    # saturated throughput of the batch solver on the stream's pairs
    sat_pairs = [r.pair for r in itertools.islice(synth.config5_requests(count=4000, rate_per_s=1e9), 4000)]
    solver.solve_batch(sat_pairs[:256], timeout_s=1.0)
    t = time.perf_counter()
    res = solver.solve_batch(sat_pairs, timeout_s=1.0)
    sat = len(sat_pairs) / (time.perf_counter() - t)
    rate = a.rate if a.rate > 0 else a.rate_frac * sat
    if a.serve_lanes:
        solver.set_serve_group(a.serve_lanes)    # before the first submit creates the server
    reqs = list(synth.config5_requests(count=n_req, rate_per_s=rate))
    # bytes each request moves: its two matrices (and labels) in, its result out
    h2d = sum(q.pair.G.n ** 2 + q.pair.H.n ** 2 + 4 * ((q.pair.G.labels is not None) * q.pair.G.n +
                                                         (q.pair.H.labels is not None) * q.pair.H.n)
              for q in reqs)
    gold = golden_sizes("c5")             # stored oracle optima of the stream's first requests
    lat, status = [], []
    out = {}
    i = 0
    t0 = time.perf_counter()
    with Clocks(0) as clk:
        while i < n_req or out:
            now = time.perf_counter() - t0
            while i < n_req and reqs[i].arrival_s <= now:
                q = reqs[i]
                tk = solver.submit(q.pair.G.adj, q.pair.H.adj, q.pair.G.labels, q.pair.H.labels,
                                   timeout_s=q.timeout_s)
                out[tk] = i
                i += 1
            done = []
            for tk, j in out.items():
                r = solver.poll(tk)
                if r is not None:
                    lat.append(time.perf_counter() - t0 - reqs[j].arrival_s)
                    status.append(r.status)
                    done.append(tk)
                    if r.status == MCS_OK and j in gold and gold[j][1] and r.size != gold[j][0]:
                        raise SystemExit(f"PARITY FAILURE request {j}: served {r.size} oracle {gold[j][0]}")
            for tk in done:
                del out[tk]
            if not done and i < n_req:
                time.sleep(max(0.0, min(2e-4, reqs[i].arrival_s - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
    lat_ms = np.array(lat) * 1e3
    solved = sum(1 for st in status if st == MCS_OK)
    # plain single-instance baseline: one pair per launch, in arrival order,
    # with the shape that suits single pairs (whole-warp searchers)
    m = min(a.single_sample, n_req)
    solver.set_launch(4, -1, 256, search_group=32)
    serv = []
    for q in reqs[:m]:
        t = time.perf_counter()
        solver.solve(q.pair.G.adj, q.pair.H.adj, q.pair.G.labels, q.pair.H.labels, timeout_s=q.timeout_s)
        serv.append(time.perf_counter() - t)
    fin, lat1 = 0.0, []
    for q, sv in zip(reqs[:m], serv):
        start = max(q.arrival_s, fin)
        fin = start + sv
        lat1.append(fin - q.arrival_s)
    lat1 = np.array(lat1) * 1e3
    line = {"metric": "MCS requests solved/sec (served, exact) on 1 B300", "value": solved / wall,
            "unit": "pairs/s", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": wall * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"Poisson stream of {n_req} requests, n log-uniform [16,56], p U[0.05,0.4], "
                                   f"0-8 labels, 1 s timeout", "rate_per_s": rate,
                       "rate_frac_of_saturated": a.rate_frac, "saturated_batch_pairs_per_s": sat,
                       "serve_lanes_per_searcher": a.serve_lanes or 32},
            "p50_latency_ms": float(np.percentile(lat_ms, 50)), "p99_latency_ms": float(np.percentile(lat_ms, 99)),
            "timeouts": sum(1 for st in status if st == MCS_TIMEOUT), "requests": len(status),
            "single_instance": {"pairs_per_s": m / sum(serv), "p50_latency_ms": float(np.percentile(lat1, 50)),
                                "p99_latency_ms": float(np.percentile(lat1, 99)), "sample": m,
                                "how": "mcs_solve per request in arrival order; FIFO queue at the same arrival times"},
            "e2e": {"value": solved / wall, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(len(status) * (24 + 2 * 64)),
                    "note": "one step = the whole stream; requests are read by the device from mapped "
                            "pinned host memory and results written back there"},
            "clocks": clk.summary()}
    solver.close()
    return line


if __name__ == "__main__":
    main()
