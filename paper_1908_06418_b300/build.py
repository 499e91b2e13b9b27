"""Builds the CUDA library ``libmcs.so`` in-tree for sm_103a (B300).

    python -m paper_1908_06418_b300.build
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmcs.so")
LIB_DEBUG = os.path.join(HERE, "libmcs_debug_bounds.so")
SOURCES = ["mcs_kernels.cu", "mcs_api.cu", "mcs_noalloc.cu", "mcs_mlp.cu", "mcs_serve.cu", "mcs_wide.cu",
           "mcs_cpu.cpp"]
HEADERS = ["mcs_internal.cuh", "mcs_cpu.h", os.path.join("..", "..", "include", "mcs.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra=None, debug: bool = False) -> str:
    """debug=True builds the MCS_DEBUG_BOUNDS variant (index checks that record
    violations instead of faulting) as libmcs_debug_bounds.so."""
    lib = LIB_DEBUG if debug else LIB
    if not force and not _stale(lib):
        return lib
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", *ARCH,
             "--expt-relaxed-constexpr"]
    if verbose:
        flags += ["-Xptxas", "-v"]
    flags += list(extra or [])
    if debug:
        flags += ["-DMCS_DEBUG_BOUNDS"]
    build_dir = os.path.join(HERE, "_build", "debug" if debug else "release")
    os.makedirs(build_dir, exist_ok=True)
    # the translation units compile in parallel (the search kernel's
    # instantiations dominate; the others overlap with it)
    from concurrent.futures import ThreadPoolExecutor
    objs = [os.path.join(build_dir, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as ex:
        jobs = [ex.submit(subprocess.check_call, [nvcc(), "-c", os.path.join(CSRC, s), "-o", o, *flags])
                for s, o in zip(SOURCES, objs)]
        for j in jobs:
            j.result()
    tmp = lib + ".tmp"
    subprocess.check_call([nvcc(), "-shared", *ARCH, *objs, "-o", tmp, "-lcudart"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
