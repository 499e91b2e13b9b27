"""The GPU + CPU race (MCS_RACE): the GPU search of a pair against a
sequential CPU McSplit of the same pair on a host thread, sharing the
incumbent through host-mapped memory; the first to finish its proof stops
the other.  Results must be exact either way: the same size with the race
on and off (and as the oracle's), with a verified mapping.  The side that
finished first is reported per solve; both sides must win somewhere on
these pairs (small pairs go to the CPU, whose start-up is cheaper, hard ones
to the GPU)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06418_b300 import Solver
    s = Solver(0)
    s.set_launch(4, -1, 256, search_group=32)       # the single-pair shape
    yield s
    s.close()


def _pairs():
    out = []
    rs = np.random.default_rng(4242)
    for i in range(24):                              # small to medium undirected and labelled pairs
        nG, nH = int(rs.integers(4, 30)), int(rs.integers(4, 30))
        k = int(rs.integers(0, 4))
        rg, rh = synth.rng_for(4242, i, 0), synth.rng_for(4242, i, 1)
        p = float(rs.uniform(0.1, 0.5))
        out.append(synth.Pair(synth.Graph(synth.er_undirected(nG, p, rg), synth.uniform_labels(nG, k, rg)),
                              synth.Graph(synth.er_undirected(nH, p, rh), synth.uniform_labels(nH, k, rh))))
    for i in range(6):                               # directed
        rg, rh = synth.rng_for(4243, i, 0), synth.rng_for(4243, i, 1)
        out.append(synth.Pair(synth.Graph(synth.er_directed(18, 0.2, rg)), synth.Graph(synth.er_directed(20, 0.2, rh)),
                              True))
    out.append(synth.config1_pair())
    out += synth.config2_pairs()[:96:24]             # hard directed pairs of 36 vertices
    return out


def test_race_is_exact_and_reports_the_winner(solver, capsys):
    from paper_1908_06418_b300 import MCS_RACE, MCS_OK
    wins = {0: 0, 1: 0, 2: 0}
    for i, p in enumerate(_pairs()):
        plain = solver.solve(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=p.directed, timeout_s=120)
        raced = solver.solve(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=p.directed, flags=MCS_RACE,
                             timeout_s=120)
        st = solver.last_stats()
        assert plain.status == MCS_OK and raced.status == MCS_OK, (i, plain.status, raced.status)
        assert raced.size == plain.size, (i, raced.size, plain.size)
        if p.G.n <= 30 or not p.directed:
            assert raced.size == oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=p.directed).size
        assert oracle.verify(p.G.adj, p.H.adj, raced.g_idx, raced.h_idx, p.G.labels, p.H.labels) == 1, i
        wins[int(st["race_winner"])] += 1
    with capsys.disabled():
        print(f"\nrace: CPU finished first on {wins[1]} pairs, GPU on {wins[2]}")
    assert wins[0] == 0
    assert wins[1] > 0 and wins[2] > 0


def test_race_time_limit_and_rejections(solver):
    from paper_1908_06418_b300 import MCS_RACE, MCS_TIMEOUT, MCS_TOP_DOWN, MCS_ERR_UNSUPPORTED
    r0, r1 = synth.rng_for(4244, 0, 0), synth.rng_for(4244, 0, 1)
    G, H = synth.er_undirected(60, 0.3, r0), synth.er_undirected(58, 0.3, r1)
    r = solver.solve(G, H, flags=MCS_RACE, timeout_s=0.3)
    assert r.status == MCS_TIMEOUT and r.size > 0
    assert oracle.verify(G, H, r.g_idx, r.h_idx) == 1
    p = synth.config1_pair()
    solver.solve_batch([p, p], flags=MCS_RACE, raise_errors=False)
    assert solver.last_rc == MCS_ERR_UNSUPPORTED                     # mcs_solve only
    with pytest.raises(RuntimeError):
        solver.solve(p.G.adj, p.H.adj, flags=MCS_RACE | MCS_TOP_DOWN)
