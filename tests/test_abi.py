"""The C-ABI library builds, loads and exports every entry point that
include/mcs.h declares (no GPU needed: no compute call is made here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mcs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcs_[a-z_]+)\s*\(", src)))


def test_header_declares_boundary():
    names = declared_functions()
    for must in ("mcs_create", "mcs_destroy", "mcs_solve", "mcs_solve_batch",
                 "mcs_solve_batch_device", "mcs_submit", "mcs_poll", "mcs_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_1908_06418_b300 as m
    lib = m.load_library()
    out = subprocess.run(["nm", "-D", "--defined-only", m.lib_path()], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (mcs_[a-z_]+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(m.EXPORTED_SYMBOLS) <= exported


def test_strerror_and_argument_checks_without_gpu():
    import paper_1908_06418_b300 as m
    lib = m.load_library()
    for code in (0, 1, 2, -1, -2, -3, -4, -5):
        assert lib.mcs_strerror(code)
    assert lib.mcs_strerror(99) == b"unknown status"
    # NULL context is rejected before any CUDA call
    assert lib.mcs_solve(None, None, None, 0, 0.0, None) == m.MCS_ERR_ARG
    assert lib.mcs_set_launch(None, 4, 0, 0) == m.MCS_ERR_ARG
    assert lib.mcs_set_search_group(None, 8) == m.MCS_ERR_ARG
    assert lib.mcs_set_steal(None, 16, 2) == m.MCS_ERR_ARG
    assert lib.mcs_set_fault(None, m.MCS_FAULT_ALLOC, 1) == m.MCS_ERR_ARG


def test_create_without_device_returns_null():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1908_06418_b300 as m
    lib = m.load_library()
    assert not lib.mcs_create(0, 0)
