"""CPU oracle for the maximum common induced subgraph problem.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA path.

* ``mcs``        -- sequential recursive McSplit (Section II-B, Algorithm 1, Eq. 1)
* ``mcs_goal``   -- one goal-directed McSplit search (Section IV-A, top-down strategy)
* ``mcs_topdown``-- the top-down strategy: goal sizes min(|V_G|,|V_H|), one less, ...
* ``mcs_deadend``-- dead-end forecasting with a bound increase and a binary search (Section IV-A)
* ``mcs_restart``-- randomized restarts over an explicit stack of pending branches (Section IV-A)
* ``hr_order`` / ``mcs_hr`` -- the static component + Hellerman-Rarick-style order (Section IV-A)
* ``bruteforce`` -- exhaustive injective partial mappings (definition, Section II-A)
* ``clique``     -- maximum clique of the modular product graph (textbook reduction)
* ``verify``     -- checks a mapping is a common induced subgraph (Section II-A)
* ``branch_log`` -- branching statistics used to train the ordering network
* ``mlp``        -- fp64 reference of the ordering network (``oracle.mlp``)

The C++ sources are compiled by ``oracle/build.py`` into
``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _b
    _b.build()                      # rebuilds only when oracle.cpp is newer
    lib = ctypes.CDLL(_LIB_PATH)
    g = [ctypes.c_int, _u8p, _i32p, ctypes.c_int, _u8p, _i32p]
    lib.oracle_verify.argtypes = g + [ctypes.c_int, _i32p, _i32p]
    lib.oracle_verify.restype = ctypes.c_int
    lib.oracle_mcs.argtypes = g + [ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                   _i32p, _i32p, _i64p, ctypes.POINTER(ctypes.c_int)]
    lib.oracle_mcs.restype = ctypes.c_int
    lib.oracle_mcs_goal.argtypes = g + [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                        ctypes.c_double, _i32p, _i32p, _i64p, ctypes.POINTER(ctypes.c_int)]
    lib.oracle_mcs_goal.restype = ctypes.c_int
    lib.oracle_mcs_topdown.argtypes = lib.oracle_mcs.argtypes
    lib.oracle_mcs_topdown.restype = ctypes.c_int
    lib.oracle_mcs_deadend.argtypes = g + [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                           ctypes.c_double, _i32p, _i32p, _i64p, ctypes.POINTER(ctypes.c_int)]
    lib.oracle_mcs_deadend.restype = ctypes.c_int
    lib.oracle_hr_order.argtypes = [ctypes.c_int, _u8p, ctypes.c_int, _i32p]
    lib.oracle_hr_order.restype = None
    lib.oracle_mcs_hr.argtypes = lib.oracle_mcs.argtypes
    lib.oracle_mcs_hr.restype = ctypes.c_int
    lib.oracle_mcs_restart.argtypes = g + [ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.c_double, _i32p, _i32p, _i64p, ctypes.POINTER(ctypes.c_int),
                                           _i64p]
    lib.oracle_mcs_restart.restype = ctypes.c_int
    lib.oracle_bruteforce.argtypes = g + [_i32p, _i32p]
    lib.oracle_bruteforce.restype = ctypes.c_int
    lib.oracle_clique.argtypes = g + [_i32p, _i32p]
    lib.oracle_clique.restype = ctypes.c_int
    lib.oracle_branch_log.argtypes = g + [ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                          _i64p, ctypes.c_int64, _i32p, _i32p,
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]
    lib.oracle_branch_log.restype = ctypes.c_int64
    lib.oracle_split_trace.argtypes = g + [ctypes.c_int, ctypes.c_int, _i32p, _i32p,
                                           _i32p, _i32p, _i32p]
    lib.oracle_split_trace.restype = ctypes.c_int
    _lib = lib
    return lib


def _gargs(adj: np.ndarray, labels: Optional[np.ndarray]):
    a = np.ascontiguousarray(adj, dtype=np.uint8)
    n = int(a.shape[0]) if a.ndim == 2 else 0
    lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.int32)
    return (n, a.ctypes.data_as(_u8p),
            (lab.ctypes.data_as(_i32p) if lab is not None else None)), (a, lab)


@dataclass
class OracleResult:
    size: int
    g_idx: np.ndarray
    h_idx: np.ndarray
    nodes: int
    complete: bool      # True iff the search finished (size proven optimal)


def mcs(adjG, adjH, labG=None, labH=None, directed: bool = False,
        node_limit: int = 0, time_limit_s: float = 0.0) -> OracleResult:
    lib = _load()
    ga, keep1 = _gargs(adjG, labG)
    ha, keep2 = _gargs(adjH, labH)
    cap = max(1, min(ga[0], ha[0]))
    og = np.zeros(cap, np.int32)
    oh = np.zeros(cap, np.int32)
    nodes = ctypes.c_int64(0)
    st = ctypes.c_int(0)
    k = lib.oracle_mcs(*ga, *ha, int(directed), int(node_limit), float(time_limit_s),
                       og.ctypes.data_as(_i32p), oh.ctypes.data_as(_i32p),
                       ctypes.byref(nodes), ctypes.byref(st))
    return OracleResult(int(k), og[:k].copy(), oh[:k].copy(), int(nodes.value), st.value == 0)


def mcs_goal(adjG, adjH, floor: int, cap: int, labG=None, labH=None, directed: bool = False,
             node_limit: int = 0, time_limit_s: float = 0.0) -> OracleResult:
    """One goal-directed search (Section IV-A): only mappings larger than
    `floor` are recorded and the search stops once one of size `cap` is
    found.  size == 0 means no mapping beat the floor; `complete` is False
    only when a limit stopped the search."""
    lib = _load()
    ga, keep1 = _gargs(adjG, labG)
    ha, keep2 = _gargs(adjH, labH)
    n = max(1, min(ga[0], ha[0]))
    og = np.zeros(n, np.int32)
    oh = np.zeros(n, np.int32)
    nodes = ctypes.c_int64(0)
    st = ctypes.c_int(0)
    k = lib.oracle_mcs_goal(*ga, *ha, int(directed), int(floor), int(cap), int(node_limit),
                            float(time_limit_s), og.ctypes.data_as(_i32p), oh.ctypes.data_as(_i32p),
                            ctypes.byref(nodes), ctypes.byref(st))
    return OracleResult(int(k), og[:k].copy(), oh[:k].copy(), int(nodes.value), st.value == 0)


def mcs_topdown(adjG, adjH, labG=None, labH=None, directed: bool = False,
                node_limit: int = 0, time_limit_s: float = 0.0) -> OracleResult:
    """The top-down strategy (Section IV-A): goal-directed searches for the goal
    sizes min(|V_G|,|V_H|), one less, ... until one is reached; `nodes` sums
    all of them."""
    lib = _load()
    ga, keep1 = _gargs(adjG, labG)
    ha, keep2 = _gargs(adjH, labH)
    n = max(1, min(ga[0], ha[0]))
    og = np.zeros(n, np.int32)
    oh = np.zeros(n, np.int32)
    nodes = ctypes.c_int64(0)
    st = ctypes.c_int(0)
    k = lib.oracle_mcs_topdown(*ga, *ha, int(directed), int(node_limit), float(time_limit_s),
                               og.ctypes.data_as(_i32p), oh.ctypes.data_as(_i32p),
                               ctypes.byref(nodes), ctypes.byref(st))
    return OracleResult(int(k), og[:k].copy(), oh[:k].copy(), int(nodes.value), st.value == 0)


def mcs_deadend(adjG, adjH, threshold: int, doubling: bool = False, labG=None, labH=None,
                directed: bool = False, node_limit: int = 0, time_limit_s: float = 0.0) -> OracleResult:
    """Dead-end forecasting (Section IV-A): the plain search raises its
    incumbent size by one (or doubles it) after `threshold` nodes without a
    new incumbent; an unreachable raised value becomes an upper bound that a
    binary search of goal-directed searches closes."""
    lib = _load()
    ga, keep1 = _gargs(adjG, labG)
    ha, keep2 = _gargs(adjH, labH)
    n = max(1, min(ga[0], ha[0]))
    og = np.zeros(n, np.int32)
    oh = np.zeros(n, np.int32)
    nodes = ctypes.c_int64(0)
    st = ctypes.c_int(0)
    k = lib.oracle_mcs_deadend(*ga, *ha, int(directed), int(threshold), int(bool(doubling)), int(node_limit),
                               float(time_limit_s), og.ctypes.data_as(_i32p), oh.ctypes.data_as(_i32p),
                               ctypes.byref(nodes), ctypes.byref(st))
    return OracleResult(int(k), og[:k].copy(), oh[:k].copy(), int(nodes.value), st.value == 0)


def hr_order(adj, directed: bool = False) -> np.ndarray:
    """The static order of Section IV-A for one graph: perm[position] = vertex."""
    lib = _load()
    a = np.ascontiguousarray(adj, dtype=np.uint8)
    n = int(a.shape[0])
    out = np.zeros(max(n, 1), np.int32)
    lib.oracle_hr_order(n, a.ctypes.data_as(_u8p), int(directed), out.ctypes.data_as(_i32p))
    return out[:n].copy()


def mcs_hr(adjG, adjH, labG=None, labH=None, directed: bool = False,
           node_limit: int = 0, time_limit_s: float = 0.0) -> OracleResult:
    """McSplit with the static order of Section IV-A instead of the degree order."""
    lib = _load()
    ga, keep1 = _gargs(adjG, labG)
    ha, keep2 = _gargs(adjH, labH)
    n = max(1, min(ga[0], ha[0]))
    og = np.zeros(n, np.int32)
    oh = np.zeros(n, np.int32)
    nodes = ctypes.c_int64(0)
    st = ctypes.c_int(0)
    k = lib.oracle_mcs_hr(*ga, *ha, int(directed), int(node_limit), float(time_limit_s),
                          og.ctypes.data_as(_i32p), oh.ctypes.data_as(_i32p),
                          ctypes.byref(nodes), ctypes.byref(st))
    return OracleResult(int(k), og[:k].copy(), oh[:k].copy(), int(nodes.value), st.value == 0)


def mcs_restart(adjG, adjH, min_nodes: int = 1, seed: int = 0, labG=None, labH=None,
                directed: bool = False, node_limit: int = 0, time_limit_s: float = 0.0):
    """Randomized restarts (Section IV-A) on an explicit stack of pending
    branches; returns (OracleResult, number of restarts)."""
    lib = _load()
    ga, keep1 = _gargs(adjG, labG)
    ha, keep2 = _gargs(adjH, labH)
    n = max(1, min(ga[0], ha[0]))
    og = np.zeros(n, np.int32)
    oh = np.zeros(n, np.int32)
    nodes = ctypes.c_int64(0)
    st = ctypes.c_int(0)
    rs = ctypes.c_int64(0)
    k = lib.oracle_mcs_restart(*ga, *ha, int(directed), int(min_nodes), int(seed) & (2**64 - 1),
                               int(node_limit), float(time_limit_s), og.ctypes.data_as(_i32p),
                               oh.ctypes.data_as(_i32p), ctypes.byref(nodes), ctypes.byref(st), ctypes.byref(rs))
    return OracleResult(int(k), og[:k].copy(), oh[:k].copy(), int(nodes.value), st.value == 0), int(rs.value)


def bruteforce(adjG, adjH, labG=None, labH=None) -> Tuple[int, np.ndarray, np.ndarray]:
    lib = _load()
    ga, keep1 = _gargs(adjG, labG)
    ha, keep2 = _gargs(adjH, labH)
    cap = max(1, min(ga[0], ha[0]))
    og = np.zeros(cap, np.int32)
    oh = np.zeros(cap, np.int32)
    k = lib.oracle_bruteforce(*ga, *ha, og.ctypes.data_as(_i32p), oh.ctypes.data_as(_i32p))
    return int(k), og[:k].copy(), oh[:k].copy()


def clique(adjG, adjH, labG=None, labH=None) -> Tuple[int, np.ndarray, np.ndarray]:
    lib = _load()
    ga, keep1 = _gargs(adjG, labG)
    ha, keep2 = _gargs(adjH, labH)
    cap = max(1, ga[0] * ha[0])
    og = np.zeros(cap, np.int32)
    oh = np.zeros(cap, np.int32)
    k = lib.oracle_clique(*ga, *ha, og.ctypes.data_as(_i32p), oh.ctypes.data_as(_i32p))
    return int(k), og[:k].copy(), oh[:k].copy()


def verify(adjG, adjH, g_idx, h_idx, labG=None, labH=None) -> int:
    """1 if (g_idx[i] -> h_idx[i]) is a common induced subgraph, else a negative code:
    -1 size, -2 range, -3 not injective, -4 label, -5 edge, -6 self-loop."""
    lib = _load()
    ga, keep1 = _gargs(adjG, labG)
    ha, keep2 = _gargs(adjH, labH)
    g = np.ascontiguousarray(g_idx, dtype=np.int32)
    h = np.ascontiguousarray(h_idx, dtype=np.int32)
    if g.shape != h.shape:
        return -1
    return int(lib.oracle_verify(*ga, *ha, int(g.size),
                                 g.ctypes.data_as(_i32p), h.ctypes.data_as(_i32p)))


def branch_log(adjG, adjH, labG=None, labH=None, directed=False, max_depth: int = 64,
               node_limit: int = 0, max_rows: int = 1 << 20):
    """Returns (rows int64[R, 6], perm_g, perm_h, size, complete).  Row columns:
    depth, v, u (renumbered ids), nodes in the (v,u) subtree, size of a new
    incumbent found inside it or -1, rank of u among the candidates tried."""
    lib = _load()
    ga, keep1 = _gargs(adjG, labG)
    ha, keep2 = _gargs(adjH, labH)
    rows = np.zeros((max_rows, 6), np.int64)
    pg = np.zeros(max(1, ga[0]), np.int32)
    ph = np.zeros(max(1, ha[0]), np.int32)
    size = ctypes.c_int(0)
    st = ctypes.c_int(0)
    r = lib.oracle_branch_log(*ga, *ha, int(directed), int(max_depth), int(node_limit),
                              rows.ctypes.data_as(_i64p), int(max_rows),
                              pg.ctypes.data_as(_i32p), ph.ctypes.data_as(_i32p),
                              ctypes.byref(size), ctypes.byref(st))
    return rows[:r].copy(), pg[:ga[0]].copy(), ph[:ha[0]].copy(), int(size.value), st.value == 0


def split_trace(adjG, adjH, g_seq, h_seq, labG=None, labH=None, directed=False):
    """Applies the oracle's class split for each pair in turn (no renumbering).
    Returns (bounds[k], cls_g[k, nG], cls_h[k, nH]) -- see oracle_split_trace."""
    lib = _load()
    ga, keep1 = _gargs(adjG, labG)
    ha, keep2 = _gargs(adjH, labH)
    gs = np.ascontiguousarray(g_seq, dtype=np.int32)
    hs = np.ascontiguousarray(h_seq, dtype=np.int32)
    k = int(gs.size)
    b = np.zeros(max(1, k), np.int32)
    cg = np.zeros((max(1, k), max(1, ga[0])), np.int32)
    ch = np.zeros((max(1, k), max(1, ha[0])), np.int32)
    lib.oracle_split_trace(*ga, *ha, int(directed), k, gs.ctypes.data_as(_i32p),
                           hs.ctypes.data_as(_i32p), b.ctypes.data_as(_i32p),
                           cg.ctypes.data_as(_i32p), ch.ctypes.data_as(_i32p))
    return b[:k], cg[:k, :ga[0]], ch[:k, :ha[0]]
