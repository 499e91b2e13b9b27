"""B300-native exact maximum common induced subgraph search (McSplit).

Thin ctypes binding over ``libmcs.so`` (C ABI in ``include/mcs.h``).  This
module only marshals arguments: validation of graph contents, renumbering,
packing, the branch and bound, and result decoding all run in the library's
CUDA kernels.  There is no CPU fallback: if the library is missing the import
of :class:`Solver` fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

__all__ = ["Solver", "Result", "MCS_OK", "MCS_TIMEOUT", "MCS_PENDING", "MCS_ERR_ARG",
           "MCS_ERR_NOMEM", "MCS_ERR_CUDA", "MCS_ERR_DEVICE_STALL", "MCS_ERR_UNSUPPORTED",
           "MCS_DIRECTED", "MCS_ORDER_LEARNED", "MCS_NO_MAPPING", "MCS_NO_LEVEL_PRUNE",
           "MCS_MAX_N", "MCS_GRAPH_REPLAY", "MCS_WIDE", "MCS_RACE", "MCS_MODE_FREE", "MCS_MODE_LOCKSTEP", "MCS_FAULT_ALLOC", "MCS_FAULT_CUDA", "MCS_FAULT_STALL_MS",
           "MCS_FAULT_SPIN_LIMIT", "MCS_FAULT_WITHHOLD_EXIT", "MCS_FAULT_BLOCK_RING", "MCS_WORD32", "MCS_TOP_DOWN", "MCS_DEAD_END", "MCS_ORDER_HR", "MCS_RESTART", "lib_path", "load_library", "EXPORTED_SYMBOLS",
           "DeviceBatch", "HostBatch", "pack_host"]

MCS_MAX_N = 256      # vertices per graph; also the stride of the device mapping outputs
MCS_OK, MCS_TIMEOUT, MCS_PENDING = 0, 1, 2
MCS_ERR_ARG, MCS_ERR_NOMEM, MCS_ERR_CUDA, MCS_ERR_DEVICE_STALL, MCS_ERR_UNSUPPORTED = -1, -2, -3, -4, -5
MCS_DIRECTED, MCS_ORDER_LEARNED, MCS_NO_MAPPING, MCS_NO_LEVEL_PRUNE = 0x1, 0x2, 0x4, 0x8
MCS_WORD32 = 0x20
MCS_TOP_DOWN = 0x40
MCS_DEAD_END = 0x80
MCS_ORDER_HR = 0x100
MCS_RESTART = 0x200
MCS_GRAPH_REPLAY = 0x10
MCS_WIDE = 0x400     # mcs_solve_batch_device: graphs of more than 64 vertices
MCS_RACE = 0x800     # mcs_solve: GPU search raced against a CPU McSplit
MCS_MODE_FREE, MCS_MODE_LOCKSTEP = 0, 1     # mcs_set_search_mode
# failure-injection kinds of mcs_set_fault (test hooks)
MCS_FAULT_ALLOC, MCS_FAULT_CUDA, MCS_FAULT_STALL_MS = 1, 2, 3
MCS_FAULT_SPIN_LIMIT, MCS_FAULT_WITHHOLD_EXIT, MCS_FAULT_BLOCK_RING = 4, 5, 6

_HERE = os.path.dirname(os.path.abspath(__file__))


def lib_path() -> str:
    return os.path.join(_HERE, "libmcs.so")


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("adj", ctypes.POINTER(ctypes.c_uint8)),
                ("labels", ctypes.POINTER(ctypes.c_int32))]


class _Result(ctypes.Structure):
    _fields_ = [("size", ctypes.c_int32), ("status", ctypes.c_int32),
                ("npairs", ctypes.c_int32), ("_pad", ctypes.c_int32),
                ("g_idx", ctypes.POINTER(ctypes.c_int16)),
                ("h_idx", ctypes.POINTER(ctypes.c_int16)),
                ("nodes", ctypes.c_uint64), ("seconds", ctypes.c_double)]


EXPORTED_SYMBOLS = ["mcs_create", "mcs_destroy", "mcs_solve", "mcs_solve_batch",
                    "mcs_solve_batch_device", "mcs_submit", "mcs_poll", "mcs_set_launch",
                    "mcs_set_max_warps", "mcs_set_search_group", "mcs_set_serve_group", "mcs_set_steal",
                    "mcs_set_dead_end", "mcs_set_restart", "mcs_set_fault", "mcs_set_search_mode",
                    "mcs_last_stats", "mcs_bench_popc", "mcs_strerror", "mcs_error_detail",
                    "mcs_solve_batch_noalloc", "mcs_set_order_model", "mcs_get_order_model",
                    "mcs_order_eval", "mcs_order_train", "mcs_order_score_grid"]

MCS_ORDER_NPARAMS = 22913

_lib = None


def load_library():
    """Loads libmcs.so (building it if the sources are newer) and declares the
    signatures.  Raises if the library cannot be built or loaded."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _b
    # MCS_DEBUG_BOUNDS=1 selects the index-checking diagnostic build
    path = _b.build(debug=os.environ.get("MCS_DEBUG_BOUNDS") == "1")
    lib = ctypes.CDLL(path)
    vp, i32, u32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_double
    gp, rp = ctypes.POINTER(_Graph), ctypes.POINTER(_Result)
    lib.mcs_create.argtypes = [ctypes.c_int, u32]
    lib.mcs_create.restype = vp
    lib.mcs_destroy.argtypes = [vp]
    lib.mcs_destroy.restype = None
    lib.mcs_solve.argtypes = [vp, gp, gp, u32, dbl, rp]
    lib.mcs_solve.restype = ctypes.c_int
    lib.mcs_solve_batch.argtypes = [vp, gp, gp, i32, u32, dbl, rp]
    lib.mcs_solve_batch.restype = ctypes.c_int
    lib.mcs_solve_batch_device.argtypes = [vp, i32, vp, vp, vp, vp, vp, u32, dbl,
                                           vp, vp, vp, vp, vp, vp]
    lib.mcs_solve_batch_device.restype = ctypes.c_int
    lib.mcs_submit.argtypes = [vp, gp, gp, u32, dbl, ctypes.POINTER(ctypes.c_uint64)]
    lib.mcs_submit.restype = ctypes.c_int
    lib.mcs_poll.argtypes = [vp, ctypes.c_uint64, rp]
    lib.mcs_poll.restype = ctypes.c_int
    lib.mcs_set_launch.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.mcs_set_launch.restype = ctypes.c_int
    lib.mcs_set_max_warps.argtypes = [vp, ctypes.c_int]
    lib.mcs_set_max_warps.restype = ctypes.c_int
    lib.mcs_set_dead_end.argtypes = [vp, ctypes.c_longlong, ctypes.c_int]
    lib.mcs_set_dead_end.restype = ctypes.c_int
    lib.mcs_set_restart.argtypes = [vp, ctypes.c_longlong, ctypes.c_ulonglong]
    lib.mcs_set_restart.restype = ctypes.c_int
    lib.mcs_set_search_mode.argtypes = [vp, ctypes.c_int]
    lib.mcs_set_search_mode.restype = ctypes.c_int
    lib.mcs_set_fault.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
    lib.mcs_set_fault.restype = ctypes.c_int
    lib.mcs_set_search_group.argtypes = [vp, ctypes.c_int]
    lib.mcs_set_search_group.restype = ctypes.c_int
    lib.mcs_set_serve_group.argtypes = [vp, ctypes.c_int]
    lib.mcs_set_serve_group.restype = ctypes.c_int
    lib.mcs_set_steal.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.mcs_set_steal.restype = ctypes.c_int
    lib.mcs_last_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    lib.mcs_last_stats.restype = ctypes.c_int
    lib.mcs_bench_popc.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.mcs_bench_popc.restype = ctypes.c_int
    lib.mcs_solve_batch_noalloc.argtypes = [i32, vp, vp, vp, vp, vp, u32, dbl,
                                            vp, vp, vp, vp, vp, vp]
    lib.mcs_solve_batch_noalloc.restype = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    lib.mcs_set_order_model.argtypes = [vp, fp, i32]
    lib.mcs_set_order_model.restype = ctypes.c_int
    lib.mcs_get_order_model.argtypes = [vp, fp, i32]
    lib.mcs_get_order_model.restype = ctypes.c_int
    lib.mcs_order_eval.argtypes = [vp, i32, vp, vp, vp, vp, vp, u32, i32, vp, vp, vp,
                                   fp, fp, fp, fp]
    lib.mcs_order_eval.restype = ctypes.c_int
    lib.mcs_order_train.argtypes = [vp, i32, vp, vp, vp, vp, vp, u32, i32, vp, vp, vp,
                                    i32, i32, ctypes.c_float, ctypes.c_uint64, fp]
    lib.mcs_order_train.restype = ctypes.c_int
    lib.mcs_order_score_grid.argtypes = [vp, i32, vp, vp, vp, vp, vp, u32, vp, vp]
    lib.mcs_order_score_grid.restype = ctypes.c_int
    lib.mcs_error_detail.argtypes = []
    lib.mcs_error_detail.restype = ctypes.c_char_p
    lib.mcs_strerror.argtypes = [ctypes.c_int]
    lib.mcs_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


@dataclass
class Result:
    size: int
    status: int
    g_idx: np.ndarray
    h_idx: np.ndarray
    nodes: int
    seconds: float


class _Keep:
    """Holds numpy buffers alive while ctypes structs point into them."""

    def __init__(self):
        self.items = []

    def graph(self, adj, labels) -> _Graph:
        a = np.ascontiguousarray(adj, dtype=np.uint8)
        n = int(a.shape[0]) if a.ndim == 2 else 0
        self.items.append(a)
        g = _Graph()
        g.n = n
        g.adj = a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        if labels is not None:
            lab = np.ascontiguousarray(labels, dtype=np.int32)
            self.items.append(lab)
            g.labels = lab.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        return g


class Solver:
    """One library context (one CUDA stream, grow-only device arenas)."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        self.ctx = self.lib.mcs_create(int(device), 0)
        if not self.ctx:
            raise RuntimeError("mcs_create failed (no CUDA device?)")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mcs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configuration ----------------------------------------------------
    def set_launch(self, warps_per_block=0, blocks_per_sm=0, smem_stack_entries=0, search_group=None):
        """0 keeps a value, -1 restores its default; search_group (lanes per
        searcher: 32, 16, 8, 4 or 2) is left alone when None."""
        rc = self.lib.mcs_set_launch(self.ctx, warps_per_block, blocks_per_sm, smem_stack_entries)
        if rc:
            raise ValueError(self.strerror(rc))
        if search_group is not None:
            self.set_search_group(search_group)

    def reset_launch(self):
        """Back to the default launch shape, search group (8 lanes) and work
        sharing."""
        self.set_launch(-1, -1, -1, search_group=8)
        self.set_steal(-1, -1)

    def set_serve_group(self, lanes: int):
        """Lanes per searcher of the server (32, 16 or 8); before the first submit."""
        rc = self.lib.mcs_set_serve_group(self.ctx, int(lanes))
        if rc:
            raise ValueError(self.strerror(rc))

    def set_steal(self, poll_nodes: int = 0, keep_quarters: int = 0):
        """Work-sharing poll interval (nodes) and the donor's kept share in
        quarters; 0 keeps a value, -1 restores its default."""
        rc = self.lib.mcs_set_steal(self.ctx, int(poll_nodes), int(keep_quarters))
        if rc:
            raise ValueError(self.strerror(rc))

    def set_max_warps(self, warps: int):
        rc = self.lib.mcs_set_max_warps(self.ctx, int(warps))
        if rc:
            raise ValueError(self.strerror(rc))

    def set_dead_end(self, threshold_nodes: int = -1, doubling: int = -1):
        """MCS_DEAD_END parameters: nodes without a new incumbent before the
        incumbent size is raised (-1: default 2^22), and whether it doubles
        (1) or adds one (0; -1: default)."""
        rc = self.lib.mcs_set_dead_end(self.ctx, int(threshold_nodes), int(doubling))
        if rc:
            raise ValueError(f"mcs_set_dead_end: {self.strerror(rc)}")

    def set_restart(self, min_nodes: int = -1, seed: int = 0):
        """MCS_RESTART parameters: nodes of a pair before its first restart
        (-1: default 2^20) and the seed of the random branch order."""
        rc = self.lib.mcs_set_restart(self.ctx, int(min_nodes), int(seed) & (2**64 - 1))
        if rc:
            raise ValueError(f"mcs_set_restart: {self.strerror(rc)}")

    def set_search_mode(self, mode: int):
        """MCS_MODE_FREE (default) or MCS_MODE_LOCKSTEP: how searchers
        narrower than a warp share it in plain batch solves."""
        rc = self.lib.mcs_set_search_mode(self.ctx, int(mode))
        if rc:
            raise ValueError(self.strerror(rc))

    def set_fault(self, kind: int, value: int):
        """Failure injection (mcs_set_fault): MCS_FAULT_* kind, value 0 = off."""
        rc = self.lib.mcs_set_fault(self.ctx, int(kind), int(value))
        if rc:
            raise ValueError(f"mcs_set_fault: {self.strerror(rc)}")

    def clear_faults(self):
        for k in (MCS_FAULT_ALLOC, MCS_FAULT_CUDA, MCS_FAULT_STALL_MS, MCS_FAULT_SPIN_LIMIT,
                  MCS_FAULT_WITHHOLD_EXIT, MCS_FAULT_BLOCK_RING):
            self.set_fault(k, 0)

    def set_search_group(self, lanes: int):
        """Lanes per searcher: 32 (one search per warp), 16, 8, 4 or 2."""
        rc = self.lib.mcs_set_search_group(self.ctx, int(lanes))
        if rc:
            raise ValueError(self.strerror(rc))

    def apply_tuned(self, pairs, directed: bool = False, cache: Optional[dict] = None) -> Optional[dict]:
        """Sets the launch shape that the autotuner recorded for the batch's
        bucket (see autotune.py); returns it, or None when none is cached."""
        from . import autotune
        c = autotune.load_cache() if cache is None else cache
        e = c.get(autotune.bucket(pairs, directed))
        if e:
            self.set_launch(e["warps_per_block"], e["blocks_per_sm"] or -1, e["smem_stack_entries"],
                            search_group=e.get("search_group", 32))
            self.set_steal(e.get("poll_nodes", -1), e.get("steal_keep_quarters", -1))
        return e

    def last_stats(self) -> dict:
        buf = (ctypes.c_double * 17)()
        self.lib.mcs_last_stats(self.ctx, buf, 17)
        return dict(kernel_us=buf[0], nodes=buf[1], donated=buf[2], stolen=buf[3],
                    spilled=buf[4], warps=buf[5], h2d_bytes=buf[6], d2h_bytes=buf[7],
                    class_visits=buf[8], pruned=buf[9], busy_cycles=buf[10],
                    idle_cycles=buf[11], dbg_count=buf[12], dbg_code=buf[13],
                    dbg_line=buf[14], race_winner=buf[15], race_cpu_nodes=buf[16])

    def bench_popc(self) -> float:
        """Measured device-wide 32-bit popcount rate (per second)."""
        out = ctypes.c_double(0)
        rc = self.lib.mcs_bench_popc(self.ctx, ctypes.byref(out))
        if rc:
            raise RuntimeError(self.strerror(rc))
        return out.value

    def strerror(self, code: int) -> str:
        return self.lib.mcs_strerror(int(code)).decode()

    # -- solving ----------------------------------------------------------
    def solve_batch(self, pairs: Sequence, flags: int = 0, timeout_s: float = 0.0,
                    directed: Optional[bool] = None, raise_errors: bool = True) -> List[Result]:
        """pairs: sequence of (adjG, adjH, labG, labH) tuples or objects with
        .G.adj/.G.labels/.H.adj/.H.labels (and optionally .directed).  The
        call's return code is kept in ``last_rc``; with raise_errors=False an
        error code other than MCS_ERR_ARG is returned there instead of raised."""
        keep = _Keep()
        n = len(pairs)
        Gs = (_Graph * max(n, 1))()
        Hs = (_Graph * max(n, 1))()
        Rs = (_Result * max(n, 1))()
        caps = []
        for i, p in enumerate(pairs):
            if hasattr(p, "G"):
                aG, aH, lG, lH = p.G.adj, p.H.adj, p.G.labels, p.H.labels
                if directed is None and getattr(p, "directed", False):
                    flags |= MCS_DIRECTED
            else:
                aG, aH, lG, lH = p
            Gs[i] = keep.graph(aG, lG)
            Hs[i] = keep.graph(aH, lH)
            cap = max(1, min(Gs[i].n, Hs[i].n))
            gi = np.zeros(cap, np.int16)
            hi = np.zeros(cap, np.int16)
            caps.append((gi, hi))
            Rs[i].g_idx = gi.ctypes.data_as(ctypes.POINTER(ctypes.c_int16))
            Rs[i].h_idx = hi.ctypes.data_as(ctypes.POINTER(ctypes.c_int16))
        if directed:
            flags |= MCS_DIRECTED
        rc = self.lib.mcs_solve_batch(self.ctx, Gs, Hs, n, flags, float(timeout_s), Rs)
        self.last_rc = int(rc)
        if rc < 0 and rc not in (MCS_ERR_ARG,) and raise_errors:
            raise RuntimeError(f"mcs_solve_batch: {self.strerror(rc)} ({rc}): "
                               f"{self.lib.mcs_error_detail().decode()}")
        out = []
        for i in range(n):
            r = Rs[i]
            k = r.npairs
            gi, hi = caps[i]
            out.append(Result(int(r.size), int(r.status), gi[:k].astype(np.int32),
                              hi[:k].astype(np.int32), int(r.nodes), float(r.seconds)))
        return out

    def solve_host(self, batch: "HostBatch", flags: int = 0, timeout_s: float = 0.0) -> dict:
        """mcs_solve_batch on a HostBatch: the same C call as solve_batch
        (host buffers; one host-to-device and one device-to-host copy inside)
        without per-pair Python objects.  Returns numpy arrays: size, status,
        nodes, seconds, and the mapping as g_idx/h_idx rows (the first size[i]
        entries of row i)."""
        gp, rp = ctypes.POINTER(_Graph), ctypes.POINTER(_Result)
        rc = self.lib.mcs_solve_batch(self.ctx, ctypes.cast(batch.G.ctypes.data, gp),
                                      ctypes.cast(batch.H.ctypes.data, gp), batch.npairs,
                                      int(flags | batch.flags), float(timeout_s),
                                      ctypes.cast(batch.res.ctypes.data, rp))
        if rc < 0 and rc not in (MCS_ERR_ARG,):
            raise RuntimeError(f"mcs_solve_batch: {self.strerror(rc)} ({rc}): "
                               f"{self.lib.mcs_error_detail().decode()}")
        k = batch.npairs
        r = batch.res[:k]
        return dict(size=r["size"].copy(), status=r["status"].copy(), nodes=r["nodes"].copy(),
                    seconds=r["seconds"].copy(), g_idx=batch.map_g[:k], h_idx=batch.map_h[:k])

    def solve(self, adjG, adjH, labG=None, labH=None, directed: bool = False,
              flags: int = 0, timeout_s: float = 0.0) -> Result:
        """One pair through mcs_solve (the entry point that also takes MCS_RACE)."""
        keep = _Keep()
        G = keep.graph(adjG, labG)
        H = keep.graph(adjH, labH)
        cap = max(1, min(G.n, H.n))
        gi = np.zeros(cap, np.int16)
        hi = np.zeros(cap, np.int16)
        r = _Result()
        r.g_idx = gi.ctypes.data_as(ctypes.POINTER(ctypes.c_int16))
        r.h_idx = hi.ctypes.data_as(ctypes.POINTER(ctypes.c_int16))
        rc = self.lib.mcs_solve(self.ctx, ctypes.byref(G), ctypes.byref(H),
                                int(flags | (MCS_DIRECTED if directed else 0)), float(timeout_s), ctypes.byref(r))
        self.last_rc = int(rc)
        if rc < 0 and rc != MCS_ERR_ARG:
            raise RuntimeError(f"mcs_solve: {self.strerror(rc)} ({rc}): {self.lib.mcs_error_detail().decode()}")
        k = r.npairs
        return Result(int(r.size), int(r.status), gi[:k].astype(np.int32), hi[:k].astype(np.int32),
                      int(r.nodes), float(r.seconds))

    # -- branching-order network -----------------------------------------
    def set_order_model(self, params: np.ndarray):
        p = np.ascontiguousarray(params, dtype=np.float32)
        rc = self.lib.mcs_set_order_model(self.ctx, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                          int(p.size))
        if rc:
            raise ValueError(f"mcs_set_order_model: {self.strerror(rc)}")

    def get_order_model(self) -> np.ndarray:
        p = np.zeros(MCS_ORDER_NPARAMS, np.float32)
        rc = self.lib.mcs_get_order_model(self.ctx, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                          int(p.size))
        if rc:
            raise ValueError(f"mcs_get_order_model: {self.strerror(rc)}")
        return p

    def order_eval(self, batch: "DeviceBatch", rows=None, y=None, w=None, scores=False,
                   loss_grad=False, features=False) -> dict:
        """rows: int32 [R, 3] (pair, v, u) in original ids; y, w: float32 [R]."""
        import torch
        fptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if a is not None else None
        dev = batch.device
        d_rows = torch.from_numpy(np.ascontiguousarray(rows, np.int32)).to(dev) if rows is not None else None
        d_y = torch.from_numpy(np.ascontiguousarray(y, np.float32)).to(dev) if y is not None else None
        d_w = torch.from_numpy(np.ascontiguousarray(w, np.float32)).to(dev) if w is not None else None
        R = 0 if rows is None else len(rows)
        out = {}
        h_s = np.zeros(max(R, 1), np.float32) if scores else None
        h_l = np.zeros(1, np.float32) if loss_grad else None
        h_g = np.zeros(MCS_ORDER_NPARAMS, np.float32) if loss_grad else None
        h_f = np.zeros((batch.npairs, 2, 64, 18), np.float32) if features else None
        ptr = _ptr
        rc = self.lib.mcs_order_eval(self.ctx, batch.npairs, ptr(batch.d_n), ptr(batch.d_adj_off),
                                     ptr(batch.d_adj), ptr(batch.d_lab_off), ptr(batch.d_labels),
                                     batch.flags, R, ptr(d_rows), ptr(d_y), ptr(d_w),
                                     fptr(h_s), fptr(h_l), fptr(h_g), fptr(h_f))
        if rc:
            raise RuntimeError(f"mcs_order_eval: {self.strerror(rc)}")
        if scores:
            out["scores"] = h_s[:R]
        if loss_grad:
            out["loss"] = float(h_l[0])
            out["grad"] = h_g
        if features:
            out["features"] = h_f
        return out

    def order_score_grid(self, batch: "DeviceBatch", out=None, stream=None):
        """Scores of every candidate pair: a float32 tensor [npairs, 64, 64]
        on the batch's device, entry [p, v, u] valid for v < n_G and u < n_H
        (the rest is left as it was).  Asynchronous on `stream` (a
        torch.cuda.Stream or a raw handle; None = the context's stream)."""
        import torch
        if out is None:
            out = torch.zeros((batch.npairs, 64, 64), dtype=torch.float32, device=batch.device)
        h = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        rc = self.lib.mcs_order_score_grid(self.ctx, batch.npairs, _ptr(batch.d_n), _ptr(batch.d_adj_off),
                                           _ptr(batch.d_adj), _ptr(batch.d_lab_off), _ptr(batch.d_labels),
                                           batch.flags, _ptr(out), h)
        if rc:
            raise RuntimeError(f"mcs_order_score_grid: {self.strerror(rc)}")
        return out

    def order_train(self, batch: "DeviceBatch", rows, y, w=None, steps=100, batch_size=4096,
                    lr=1e-3, seed=1) -> np.ndarray:
        import torch
        dev = batch.device
        d_rows = torch.from_numpy(np.ascontiguousarray(rows, np.int32)).to(dev)
        d_y = torch.from_numpy(np.ascontiguousarray(y, np.float32)).to(dev)
        d_w = torch.from_numpy(np.ascontiguousarray(w, np.float32)).to(dev) if w is not None else None
        losses = np.zeros(max(steps, 1), np.float32)
        rc = self.lib.mcs_order_train(self.ctx, batch.npairs, _ptr(batch.d_n), _ptr(batch.d_adj_off),
                                      _ptr(batch.d_adj), _ptr(batch.d_lab_off), _ptr(batch.d_labels),
                                      batch.flags, len(rows), _ptr(d_rows), _ptr(d_y), _ptr(d_w),
                                      int(steps), int(batch_size), float(lr), int(seed),
                                      losses.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if rc:
            raise RuntimeError(f"mcs_order_train: {self.strerror(rc)}")
        return losses[:steps]

    # -- serving ---------------------------------------------------------
    def submit(self, adjG, adjH, labG=None, labH=None, flags: int = 0,
               timeout_s: float = 1.0) -> int:
        """Admits one request (undirected); returns its ticket.  The graphs are
        copied before the call returns."""
        keep = _Keep()
        G = keep.graph(adjG, labG)
        H = keep.graph(adjH, labH)
        t = ctypes.c_uint64(0)
        rc = self.lib.mcs_submit(self.ctx, ctypes.byref(G), ctypes.byref(H), int(flags),
                                 float(timeout_s), ctypes.byref(t))
        if rc < 0:
            raise RuntimeError(f"mcs_submit: {self.strerror(rc)} ({rc})")
        return int(t.value)

    def poll(self, ticket: int, raise_errors: bool = True) -> Optional[Result]:
        """None while the request runs; its Result once finished (the ticket is
        then released).  A request lost by a failed server launch raises, or
        with raise_errors=False returns a Result whose status is the error."""
        gi = np.zeros(MCS_MAX_N, np.int16)
        hi = np.zeros(MCS_MAX_N, np.int16)
        r = _Result()
        r.g_idx = gi.ctypes.data_as(ctypes.POINTER(ctypes.c_int16))
        r.h_idx = hi.ctypes.data_as(ctypes.POINTER(ctypes.c_int16))
        rc = self.lib.mcs_poll(self.ctx, ctypes.c_uint64(int(ticket)), ctypes.byref(r))
        if rc == MCS_PENDING:
            return None
        if rc < 0 and rc != MCS_ERR_ARG and raise_errors:
            raise RuntimeError(f"mcs_poll: {self.strerror(rc)} ({rc})")
        if rc == MCS_ERR_ARG and r.status == 0 and r.size == 0:
            raise KeyError(f"unknown ticket {ticket}")
        k = r.npairs
        return Result(int(r.size), int(r.status), gi[:k].astype(np.int32), hi[:k].astype(np.int32),
                      int(r.nodes), float(r.seconds))

    def solve_batch_device(self, npairs: int, d_n, d_adj_off, d_adj, d_lab_off, d_labels,
                           d_size, d_status, d_nodes, d_map=None, d_usec=None, flags: int = 0,
                           timeout_s: float = 0.0, stream: int = 0) -> int:
        """Device-resident batch: every argument is a torch CUDA tensor (or None)
        in the layout documented for mcs_solve_batch_device; nothing is copied
        and nothing is synchronised.  Returns the enqueue status."""
        def ptr(t):
            return None if t is None else ctypes.c_void_p(int(t.data_ptr()))
        return int(self.lib.mcs_solve_batch_device(
            self.ctx, int(npairs), ptr(d_n), ptr(d_adj_off), ptr(d_adj), ptr(d_lab_off),
            ptr(d_labels), int(flags), float(timeout_s), ptr(d_size), ptr(d_status),
            ptr(d_nodes), ptr(d_map), ptr(d_usec),
            ctypes.c_void_p(int(stream)) if stream else None))


def pack_host(pairs) -> dict:
    """Lays a list of pairs out in the flat format of mcs_solve_batch_device
    (numpy arrays; the caller moves them to the device).  Argument marshalling
    only: no graph arithmetic happens here."""
    n, adj_off, lab_off, blobs, labs = [], [], [], [], []
    ao = lo = 0
    for p in pairs:
        for g in (p.G, p.H):
            a = np.ascontiguousarray(g.adj, dtype=np.uint8).reshape(-1)
            n.append(int(g.adj.shape[0]))
            adj_off.append(ao)
            blobs.append(a)
            ao += a.size
            if g.labels is not None:
                lab_off.append(lo)
                labs.append(np.ascontiguousarray(g.labels, dtype=np.int32))
                lo += len(g.labels)
            else:
                lab_off.append(-1)
    return dict(
        n=np.asarray(n, np.int32), adj_off=np.asarray(adj_off, np.int64),
        adj=np.concatenate(blobs) if blobs else np.zeros(16, np.uint8),
        lab_off=np.asarray(lab_off, np.int64),
        labels=np.concatenate(labs) if labs else None)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(int(t.data_ptr()))


# numpy images of mcs_graph / mcs_result (include/mcs.h), for whole-batch marshalling
_GRAPH_DTYPE = np.dtype([("n", "<i4"), ("_pad", "<i4"), ("adj", "<u8"), ("labels", "<u8")])
_RESULT_DTYPE = np.dtype([("size", "<i4"), ("status", "<i4"), ("npairs", "<i4"), ("_pad", "<i4"),
                          ("g_idx", "<u8"), ("h_idx", "<u8"), ("nodes", "<u8"), ("seconds", "<f8")])
assert _GRAPH_DTYPE.itemsize == ctypes.sizeof(_Graph) and _RESULT_DTYPE.itemsize == ctypes.sizeof(_Result)


class HostBatch:
    """A list of pairs in host memory, laid out once for mcs_solve_batch
    (Solver.solve_host): the mcs_graph arrays point into one adjacency buffer
    and one label buffer, and the mcs_result array into one mapping buffer of
    64 entries per pair.  Marshalling only."""

    def __init__(self, pairs, directed: bool = False):
        h = pack_host(pairs)
        self.npairs = len(pairs)
        self.flags = MCS_DIRECTED if directed else 0
        self.adj = h["adj"]
        self.labels = h["labels"] if h["labels"] is not None else np.zeros(1, np.int32)
        n = h["n"]
        g = np.zeros(2 * max(self.npairs, 1), _GRAPH_DTYPE)
        g["n"][:n.size] = n
        g["adj"][:n.size] = self.adj.ctypes.data + h["adj_off"]
        lo = h["lab_off"]
        g["labels"][:n.size] = np.where(lo >= 0, self.labels.ctypes.data + 4 * np.maximum(lo, 0), 0)
        self.G = np.ascontiguousarray(g[0::2])
        self.H = np.ascontiguousarray(g[1::2])
        self.map_g = np.zeros((max(self.npairs, 1), MCS_MAX_N), np.int16)
        self.map_h = np.zeros((max(self.npairs, 1), MCS_MAX_N), np.int16)
        self.res = np.zeros(max(self.npairs, 1), _RESULT_DTYPE)
        self.res["g_idx"] = self.map_g.ctypes.data + 2 * MCS_MAX_N * np.arange(self.res.size)
        self.res["h_idx"] = self.map_h.ctypes.data + 2 * MCS_MAX_N * np.arange(self.res.size)


class DeviceBatch:
    """A list of pairs laid out for the device entry points (torch tensors
    hold the device memory; flags carries MCS_DIRECTED when the pairs are
    directed, MCS_WORD32 when every graph has at most 32 vertices unless
    word32=False, and MCS_WIDE when a graph has more than 64)."""

    def __init__(self, pairs, device=0, directed: bool = False, word32: Optional[bool] = None):
        import torch
        h = pack_host(pairs)
        self.device = torch.device("cuda", device) if isinstance(device, int) else device
        self.npairs = len(pairs)
        self.flags = MCS_DIRECTED if directed else 0
        fits = len(pairs) > 0 and all(p.G.n <= 32 and p.H.n <= 32 for p in pairs)
        if word32 is None:
            word32 = fits
        if word32:
            self.flags |= MCS_WORD32
        if any(max(p.G.n, p.H.n) > 64 for p in pairs):
            self.flags |= MCS_WIDE
        self.d_n = torch.from_numpy(h["n"]).to(self.device)
        self.d_adj_off = torch.from_numpy(h["adj_off"]).to(self.device)
        self.d_adj = torch.from_numpy(h["adj"]).to(self.device)
        self.d_lab_off = torch.from_numpy(h["lab_off"]).to(self.device)
        self.d_labels = (torch.from_numpy(h["labels"]).to(self.device)
                         if h["labels"] is not None else None)
