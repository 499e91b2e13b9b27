"""The allocation-free batch entry point, called through the C ABI.

mcs_solve_batch_noalloc serves callers that cannot allocate device memory
(during stream capture, inside a framework that owns all device memory, or
on a latency-critical path); it keeps its scratch in a fixed device array.
This test compares it with the regular device entry point on the same inputs,
twice in a row (the second call reuses the array the first one left behind):
sizes and statuses must be identical (exact integer results), and every
mapping must be a valid common induced subgraph.  The file is named so that
pytest collects it last."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

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
                    map=torch.zeros(n * 64, dtype=torch.int16, device=dev),
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
        mp = o["map"].cpu().numpy().reshape(n, 64)
        assert (status == ref_status).all(), call
        assert (size == ref_size).all(), call
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
