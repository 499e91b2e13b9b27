"""Failure detection, tested without faulting the GPU.

Every device-side wait of the search is bounded (an idle searcher's wait for
work by a time limit without progress anywhere in the launch, a wait for a
free work-ring slot by an iteration count).  The library's failure-injection
hooks (mcs_set_fault) make such a wait run out on purpose -- an exit token
that is never posted, ring slots that never free up -- and the tests check
that the call comes back with MCS_ERR_DEVICE_STALL in bounded time, that
pairs finished before the failure keep exact results, and that the context
solves correctly afterwards.  Host-side injection makes one allocation, or
the first launch of a call, fail as if the system had refused it.  The
MCS_DEBUG_BOUNDS build (index checks that record a violation and skip the
access, in place of a sanitizer) runs small mixed batches in a child process
and must record no violation.  Nothing here traps, asserts on the device or
touches a bad address."""
import os
import subprocess
import sys
import textwrap
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def solver():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06418_b300 import Solver
    s = Solver(0)
    yield s
    s.close()


def _pairs(count, seed, directed=False, k=0, nmin=8, nmax=22):
    rs = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nG, nH = int(rs.integers(nmin, nmax + 1)), int(rs.integers(nmin, nmax + 1))
        rg, rh = synth.rng_for(seed, i, 0), synth.rng_for(seed, i, 1)
        p = float(rs.uniform(0.1, 0.5))
        if directed:
            G, H = synth.er_directed(nG, p, rg), synth.er_directed(nH, p, rh)
        else:
            G, H = synth.er_undirected(nG, p, rg), synth.er_undirected(nH, p, rh)
        out.append(synth.Pair(synth.Graph(G, synth.uniform_labels(nG, k, rg)),
                              synth.Graph(H, synth.uniform_labels(nH, k, rh)), directed))
    return out


def _oracle_sizes(pairs):
    return [oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels, directed=p.directed).size for p in pairs]


def _check_exact(pairs, res, sizes, allow_pending=False):
    from paper_1908_06418_b300 import MCS_OK, MCS_PENDING
    finished = 0
    for p, r, k in zip(pairs, res, sizes):
        if allow_pending and r.status == MCS_PENDING:
            continue
        assert r.status == MCS_OK, r.status
        assert r.size == k, (r.size, k)
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1
        finished += 1
    return finished


def test_withheld_exit_token_expires_the_idle_wait(solver):
    """The searcher that ends the batch posts one exit token too few: one
    searcher waits for work that never comes and gives up at the idle-wait
    limit (200 ms here).  Every pair was finished before that, exactly."""
    from paper_1908_06418_b300 import (MCS_ERR_DEVICE_STALL, MCS_FAULT_STALL_MS,
                                       MCS_FAULT_WITHHOLD_EXIT)
    pairs = _pairs(32, 901, k=2)
    sizes = _oracle_sizes(pairs)
    for group in (32, 8):
        solver.set_launch(4, -1, 256, search_group=group)
        solver.set_fault(MCS_FAULT_STALL_MS, 200)
        solver.set_fault(MCS_FAULT_WITHHOLD_EXIT, 1)
        t = time.time()
        res = solver.solve_batch(pairs, timeout_s=30, raise_errors=False)
        dt = time.time() - t
        assert solver.last_rc == MCS_ERR_DEVICE_STALL, solver.last_rc
        assert dt < 20.0, dt
        assert _check_exact(pairs, res, sizes) == len(pairs)
        solver.clear_faults()
        res = solver.solve_batch(pairs, timeout_s=30)
        assert solver.last_rc == 0
        _check_exact(pairs, res, sizes)
    solver.reset_launch()


@pytest.mark.parametrize("directed", [False, True])
def test_blocked_ring_expires_the_slot_wait(solver, directed):
    """Work-ring slots other than the pair roots never free up, so the first
    hand-over of work (a donation or an exit token) waits until its iteration
    limit runs out.  The call returns MCS_ERR_DEVICE_STALL; pairs that
    finished keep exact results, the rest stay MCS_PENDING (none is reported
    with a wrong size); the next call is exact."""
    from paper_1908_06418_b300 import MCS_ERR_DEVICE_STALL, MCS_FAULT_BLOCK_RING, MCS_FAULT_SPIN_LIMIT
    pairs = _pairs(24, 902 + directed, directed=directed, nmin=14, nmax=26)
    sizes = _oracle_sizes(pairs)
    solver.set_fault(MCS_FAULT_SPIN_LIMIT, 20000)
    solver.set_fault(MCS_FAULT_BLOCK_RING, 1)
    t = time.time()
    res = solver.solve_batch(pairs, timeout_s=30, raise_errors=False)
    assert time.time() - t < 30.0
    assert solver.last_rc == MCS_ERR_DEVICE_STALL, solver.last_rc
    _check_exact(pairs, res, sizes, allow_pending=True)
    solver.clear_faults()
    res = solver.solve_batch(pairs, timeout_s=30)
    assert solver.last_rc == 0
    assert _check_exact(pairs, res, sizes) == len(pairs)


def test_serving_requests_lost_by_a_failed_server_report_the_stall():
    """The server launch cannot hand requests to searchers (ring slots never
    free up): it gives up, and every request published while it ran is
    reported with MCS_ERR_DEVICE_STALL by mcs_poll instead of waiting forever.
    With the fault cleared the next request starts a fresh launch and is
    solved exactly."""
    from paper_1908_06418_b300 import (Solver, MCS_ERR_DEVICE_STALL, MCS_OK, MCS_FAULT_BLOCK_RING,
                                       MCS_FAULT_SPIN_LIMIT, MCS_FAULT_STALL_MS)
    pairs = _pairs(4, 903, k=3)
    with Solver(0) as s:
        s.set_fault(MCS_FAULT_SPIN_LIMIT, 20000)
        s.set_fault(MCS_FAULT_STALL_MS, 200)
        s.set_fault(MCS_FAULT_BLOCK_RING, 1)
        tickets = [s.submit(p.G.adj, p.H.adj, p.G.labels, p.H.labels, timeout_s=5) for p in pairs[:3]]
        got = {}
        t0 = time.time()
        while len(got) < len(tickets) and time.time() - t0 < 60:
            for tk in tickets:
                if tk not in got:
                    r = s.poll(tk, raise_errors=False)
                    if r is not None:
                        got[tk] = r
            time.sleep(0.005)
        assert len(got) == len(tickets), "polls did not finish"
        assert all(r.status == MCS_ERR_DEVICE_STALL for r in got.values()), [r.status for r in got.values()]
        s.clear_faults()
        p = pairs[3]
        tk = s.submit(p.G.adj, p.H.adj, p.G.labels, p.H.labels, timeout_s=30)
        t0 = time.time()
        r = None
        while r is None and time.time() - t0 < 60:
            r = s.poll(tk)
            time.sleep(0.002)
        assert r is not None and r.status == MCS_OK
        assert r.size == oracle.mcs(p.G.adj, p.H.adj, p.G.labels, p.H.labels).size
        assert oracle.verify(p.G.adj, p.H.adj, r.g_idx, r.h_idx, p.G.labels, p.H.labels) == 1


def test_injected_allocation_failures_leave_a_usable_context():
    """A fresh context's first batch solve makes a dozen device and pinned
    allocations.  Failing each one in turn makes that call return
    MCS_ERR_NOMEM (no crash), and the next call on the same context
    allocates again and solves exactly."""
    from paper_1908_06418_b300 import Solver, MCS_ERR_NOMEM, MCS_FAULT_ALLOC
    import paper_1908_06418_b300 as m
    pairs = _pairs(12, 904, k=2)
    sizes = _oracle_sizes(pairs)
    failed_sites = 0
    for k in range(1, 40):
        with Solver(0) as s:
            s.set_max_warps(64)
            s.set_fault(MCS_FAULT_ALLOC, k)
            res = s.solve_batch(pairs, timeout_s=30, raise_errors=False)
            if s.last_rc == 0:
                _check_exact(pairs, res, sizes)
                break
            assert s.last_rc == MCS_ERR_NOMEM, (k, s.last_rc)
            assert b"injected" in m.load_library().mcs_error_detail()
            failed_sites += 1
            res = s.solve_batch(pairs, timeout_s=30)
            assert s.last_rc == 0
            assert _check_exact(pairs, res, sizes) == len(pairs)
    assert failed_sites >= 10, failed_sites


def test_injected_cuda_error_is_reported_and_the_context_recovers(solver):
    from paper_1908_06418_b300 import MCS_ERR_CUDA, MCS_FAULT_CUDA
    import paper_1908_06418_b300 as m
    pairs = _pairs(8, 905, directed=True)
    sizes = _oracle_sizes(pairs)
    solver.set_fault(MCS_FAULT_CUDA, 2)
    for _ in range(2):
        solver.solve_batch(pairs, timeout_s=30, raise_errors=False)
        assert solver.last_rc == MCS_ERR_CUDA
        assert b"injected" in m.load_library().mcs_error_detail()
    res = solver.solve_batch(pairs, timeout_s=30)
    assert solver.last_rc == 0
    assert _check_exact(pairs, res, sizes) == len(pairs)


def test_fault_kinds_are_checked(solver):
    from paper_1908_06418_b300 import MCS_FAULT_SPIN_LIMIT
    with pytest.raises(ValueError):
        solver.set_fault(99, 1)
    with pytest.raises(ValueError):
        solver.set_fault(MCS_FAULT_SPIN_LIMIT, -1)
    with pytest.raises(ValueError):
        solver.set_fault(MCS_FAULT_SPIN_LIMIT, 1 << 33)
    solver.clear_faults()


_DEBUG_SCRIPT = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import oracle, synth
    from tests.test_gpu_faults import _pairs, _oracle_sizes, _check_exact
    from paper_1908_06418_b300 import Solver, MCS_TOP_DOWN, MCS_RESTART, lib_path
    import paper_1908_06418_b300 as m
    lib = m.load_library()
    assert lib._name.endswith("libmcs_debug_bounds.so"), lib._name
    total = 0
    with Solver(0) as s:
        # (lanes, directed, labels, flags, largest n): up to 22 vertices the
        # 32-bit node step, labelled pairs up to 40 vertices the 64-bit one
        cases = [(32, False, 0, 0, 22), (8, False, 3, 0, 40), (4, True, 0, 0, 20), (2, True, 3, 0, 40),
                 (16, False, 3, 0, 40), (8, False, 0, MCS_TOP_DOWN, 22), (4, True, 0, MCS_RESTART, 20)]
        for i, (group, directed, k, flags, nmax) in enumerate(cases):
            s.set_launch(4, -1, 64, search_group=group)
            s.set_restart(64, 5)
            pairs = _pairs(64, 950 + i, directed=directed, k=k, nmin=6, nmax=nmax)
            sizes = _oracle_sizes(pairs)
            res = s.solve_batch(pairs, flags=flags, timeout_s=60)
            st = s.last_stats()
            assert st["dbg_count"] == 0, (i, st["dbg_count"], st["dbg_code"], st["dbg_line"])
            total += _check_exact(pairs, res, sizes)
    print("DEBUG_BOUNDS_OK", total)
""")


def test_debug_bounds_build_records_no_violation():
    """The MCS_DEBUG_BOUNDS library (selected by the environment variable of
    the same name; a process loads one library) checks every stack, level,
    slot and result index.  Small mixed batches -- whole-warp, 16-, 8-, 4- and
    2-lane searchers (lockstep, the default), undirected, directed and
    labelled, both word widths, top-down and restarts -- must record no
    violation and match the oracle."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, MCS_DEBUG_BOUNDS="1")
    out = subprocess.run([sys.executable, "-c", _DEBUG_SCRIPT.format(root=ROOT)], env=env, cwd=ROOT,
                         capture_output=True, text=True, timeout=1500)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "DEBUG_BOUNDS_OK" in out.stdout
    assert int(out.stdout.split("DEBUG_BOUNDS_OK")[1].split()[0]) == 7 * 64
