"""The allocation-free batch entry point, called through the C ABI.

mcs_solve_batch_noalloc serves callers that cannot allocate device memory
(during stream capture, inside a framework that owns all device memory, or
on a latency-critical path); it keeps its scratch in a fixed device array.
The tests compare it with the regular device entry point on the same inputs,
twice in a row (the second call reuses the array the first one left behind):
sizes and statuses must be identical (exact integer results), and every
mapping must be a valid common induced subgraph.  Directed pairs, the 32-bit
node step, MCS_NO_MAPPING and the top-down strategy are checked against the
CPU oracle, and the call is captured into a CUDA graph in the capture mode
that fails on any allocation and replayed.  The file is named so that pytest
collects it last."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from paper_1908_06418_b300 import MCS_MAX_N

pytestmark = pytest.mark.gpu


def _pairs():
    rs = np.random.default_rng(2718)
    out = []
    for i in range(48):
        nG, nH = int(rs.integers(8, 30)), int(rs.integers(8, 30))
        rg, rh = synth.rng_for(271, i, 0), synth.rng_for(271, i, 1)
        out.append(synth.Pair(
            synth.Graph(synth.er_undirected(nG, float(rs.uniform(0.1, 0.5)), rg),
                        synth.uniform_labels(nG, 3, rg)),
            synth.Graph(synth.er_undirected(nH, float(rs.uniform(0.1, 0.5)), rh),
                        synth.uniform_labels(nH, 3, rh))))
    return out


def test_noalloc_matches_device_entry_point_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_06418_b300 as m
    lib = m.load_library()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pairs = _pairs()
    h = m.pack_host(pairs)
    d = {k: (torch.from_numpy(v).to(dev) if v is not None else None) for k, v in h.items()}
    n = len(pairs)

    def outs():
        return dict(size=torch.full((n,), -7, dtype=torch.int32, device=dev),
                    status=torch.full((n,), -7, dtype=torch.int32, device=dev),
                    nodes=torch.zeros(n, dtype=torch.int64, device=dev),
                    map=torch.zeros(n * MCS_MAX_N, dtype=torch.int16, device=dev),
                    usec=torch.zeros(n, dtype=torch.float32, device=dev))

    def ptr(t):
        return None if t is None else ctypes.c_void_p(int(t.data_ptr()))

    stream = torch.cuda.Stream(dev)
    with m.Solver(0) as solver:
        ref = outs()
        rc = solver.solve_batch_device(n, d["n"], d["adj_off"], d["adj"], d["lab_off"],
                                       d["labels"], ref["size"], ref["status"], ref["nodes"],
                                       ref["map"], ref["usec"], timeout_s=60,
                                       stream=stream.cuda_stream)
        assert rc == 0
        stream.synchronize()
    ref_size = ref["size"].cpu().numpy()
    ref_status = ref["status"].cpu().numpy()
    assert (ref_status == 0).all()

    for call in range(2):
        o = outs()
        rc = lib.mcs_solve_batch_noalloc(
            n, ptr(d["n"]), ptr(d["adj_off"]), ptr(d["adj"]), ptr(d["lab_off"]),
            ptr(d["labels"]), 0, 60.0, ptr(o["size"]), ptr(o["status"]), ptr(o["nodes"]),
            ptr(o["map"]), ptr(o["usec"]), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, (call, rc)
        stream.synchronize()
        size = o["size"].cpu().numpy()
        status = o["status"].cpu().numpy()
        mp = o["map"].cpu().numpy().reshape(n, MCS_MAX_N)
        assert (status == ref_status).all(), call
        assert (size == ref_size).all(), call
        for i, p in enumerate(pairs):
            g = np.nonzero(mp[i] >= 0)[0]
            assert len(g) == size[i]
            assert oracle.verify(p.G.adj, p.H.adj, g, mp[i][g], p.G.labels, p.H.labels) == 1


def _device(pairs, dev):
    import torch
    import paper_1908_06418_b300 as m
    h = m.pack_host(pairs)
    return {k: (torch.from_numpy(v).to(dev) if v is not None else None) for k, v in h.items()}


def _outs(n, dev):
    import torch
    return dict(size=torch.full((n,), -7, dtype=torch.int32, device=dev),
                status=torch.full((n,), -7, dtype=torch.int32, device=dev),
                nodes=torch.zeros(n, dtype=torch.int64, device=dev),
                map=torch.full((n * MCS_MAX_N,), -9, dtype=torch.int16, device=dev),
                usec=torch.zeros(n, dtype=torch.float32, device=dev))


def _call(lib, d, o, n, flags, stream):
    def ptr(t):
        return None if t is None else ctypes.c_void_p(int(t.data_ptr()))
    return lib.mcs_solve_batch_noalloc(n, ptr(d["n"]), ptr(d["adj_off"]), ptr(d["adj"]), ptr(d["lab_off"]),
                                       ptr(d["labels"]), flags, 60.0, ptr(o["size"]), ptr(o["status"]),
                                       ptr(o["nodes"]), ptr(o["map"]), ptr(o["usec"]),
                                       ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("case", ["directed", "directed-word32", "word32-labelled", "top-down"])
def test_noalloc_flags_match_the_oracle(case):
    """Directed pairs (4-way split), the 32-bit node step (MCS_WORD32), and
    the top-down strategy, through the allocation-free call, against the CPU
    oracle's optimum; the mapping is verified."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_06418_b300 as m
    lib = m.load_library()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rs = np.random.default_rng(31415)
    directed = case.startswith("directed")
    # unlabelled pairs of more than about 30 vertices can take the CPU oracle
    # minutes each, so the unlabelled cases stay below that
    nmax = 28 if case in ("directed", "top-down") else 32
    k = 3 if case == "word32-labelled" else 0
    pairs = []
    for i in range(40):
        nG, nH = int(rs.integers(6, nmax + 1)), int(rs.integers(6, nmax + 1))
        rg, rh = synth.rng_for(314, i, 0), synth.rng_for(314, i, 1)
        p = float(rs.uniform(0.1, 0.4))
        gen = synth.er_directed if directed else synth.er_undirected
        pairs.append(synth.Pair(synth.Graph(gen(nG, p, rg), synth.uniform_labels(nG, k, rg)),
                                synth.Graph(gen(nH, p, rh), synth.uniform_labels(nH, k, rh)), directed))
    flags = (m.MCS_DIRECTED if directed else 0) | (m.MCS_WORD32 if "word32" in case else 0) | \
            (m.MCS_TOP_DOWN if case == "top-down" else 0)
    d = _device(pairs, dev)
    stream = torch.cuda.Stream(dev)
    for call in range(2):
        o = _outs(len(pairs), dev)
        assert _call(lib, d, o, len(pairs), flags, stream) == 0
        stream.synchronize()
        size, status = o["size"].cpu().numpy(), o["status"].cpu().numpy()
        mp = o["map"].cpu().numpy().reshape(len(pairs), MCS_MAX_N)
        for i, p in enumerate(pairs):
            ref = oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=directed)
            assert status[i] == m.MCS_OK, (call, i, status[i])
            assert size[i] == ref.size, (call, i, size[i], ref.size)
            g = np.nonzero(mp[i] >= 0)[0]
            assert len(g) == size[i]
            assert oracle.verify(p.G.adj, p.H.adj, g, mp[i][g], p.G.labels, p.H.labels) == 1


def test_noalloc_no_mapping_and_learned_order():
    """MCS_NO_MAPPING leaves the mapping buffer untouched and keeps the sizes;
    the learned order (it needs a context's network) is refused with
    MCS_ERR_UNSUPPORTED before anything is enqueued."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_06418_b300 as m
    lib = m.load_library()
    dev = torch.device("cuda", 0)
    pairs = _pairs()[:16]
    d = _device(pairs, dev)
    stream = torch.cuda.Stream(dev)
    o = _outs(len(pairs), dev)
    assert _call(lib, d, o, len(pairs), m.MCS_NO_MAPPING, stream) == 0
    stream.synchronize()
    assert (o["map"].cpu().numpy() == -9).all()
    for i, p in enumerate(pairs):
        assert o["status"][i].item() == m.MCS_OK
        assert o["size"][i].item() == oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels).size
    o2 = _outs(len(pairs), dev)
    assert _call(lib, d, o2, len(pairs), m.MCS_ORDER_LEARNED, stream) == m.MCS_ERR_UNSUPPORTED
    stream.synchronize()
    assert (o2["size"].cpu().numpy() == -7).all()


def test_noalloc_captured_in_a_graph_that_forbids_allocation():
    """A caller that captures its work into a CUDA graph: the call is made
    inside torch.cuda.graph in the global capture mode, where any allocation
    (or other call that is unsafe during capture) would fail the capture.
    The first call on the device, which does the one-time set-up, happens
    before the capture.  Replays of the graph give the device entry point's
    sizes, with verified mappings, twice."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_06418_b300 as m
    lib = m.load_library()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pairs = _pairs()
    n = len(pairs)
    d = _device(pairs, dev)
    stream = torch.cuda.Stream(dev)
    warm = _outs(n, dev)
    assert _call(lib, d, warm, n, 0, stream) == 0          # set-up outside the capture
    stream.synchronize()
    ref_size = warm["size"].cpu().numpy().copy()
    with m.Solver(0) as solver:
        ref = _outs(n, dev)
        assert solver.solve_batch_device(n, d["n"], d["adj_off"], d["adj"], d["lab_off"], d["labels"],
                                         ref["size"], ref["status"], ref["nodes"], ref["map"], ref["usec"],
                                         timeout_s=60, stream=stream.cuda_stream) == 0
        stream.synchronize()
    assert (ref["size"].cpu().numpy() == ref_size).all()
    o = _outs(n, dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="global"):
        cap = torch.cuda.current_stream()
        rc = _call(lib, d, o, n, 0, cap)
    assert rc == 0
    for rep in range(2):
        o["size"].fill_(-7)
        o["status"].fill_(-7)
        graph.replay()
        torch.cuda.synchronize()
        size = o["size"].cpu().numpy()
        assert (o["status"].cpu().numpy() == m.MCS_OK).all(), rep
        assert (size == ref_size).all(), rep
        mp = o["map"].cpu().numpy().reshape(n, MCS_MAX_N)
        for i, p in enumerate(pairs):
            g = np.nonzero(mp[i] >= 0)[0]
            assert len(g) == size[i]
            assert oracle.verify(p.G.adj, p.H.adj, g, mp[i][g], p.G.labels, p.H.labels) == 1


def test_noalloc_rejects_batches_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_06418_b300 as m
    lib = m.load_library()
    too_many = 257    # MCS_NOALLOC_MAX_PAIRS + 1
    rc = lib.mcs_solve_batch_noalloc(too_many, None, None, None, None, None, 0, 1.0, None,
                                     None, None, None, None, None)
    assert rc == m.MCS_ERR_ARG
