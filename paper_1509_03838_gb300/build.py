"""Build libne.so (the CUDA library) in-tree for sm_103a with nvcc.

Translation units compile in parallel into ``_build/``; the shared library
lands next to this file so the binding (``ne.py``) loads it from the package
directory.  Rebuilds only what is older than its sources or headers.

``build(debug=True)`` makes the debug build instead: the same sources
compiled with ``-DNE_INDEX_CHECKS`` into ``_build_debug/`` and linked as
``libne_debug.so``, whose kernels check the indices of their key accesses
and record violations in a status word (``ne_debug_index_status``).  The
binding loads it in place of libne.so when ``NE_INDEX_CHECKS=1`` is set.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libne.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(HERE, "libne_debug.so")

SOURCES = ["ne_host.cpp", "ne_stream_ops.cu", "ne_conv.cu", "ne_conv_tcr_w32.cu",
           "ne_conv_tcr_w64.cu", "ne_conv_tcr_w32s.cu", "ne_conv_tcr_w64s.cu",
           "ne_conv_tcr_w32l.cu", "ne_conv_tcr_w64l.cu",
           "ne_batch.cu", "ne_gemm.cu", "ne_pipe.cu", "ne_failstop.cu"]
# the instruction-rate probe (include/ne_probe.h): a library of its own,
# used by the benchmark for its roofline denominators
PROBE_SOURCES = ["ne_probe.cu"]
PROBE_LIB = os.path.join(HERE, "libne_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-O3", f"-I{os.path.join(ROOT, 'include')}",
              "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"),
                 "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libne.so")


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
        os.path.join(ROOT, "include", "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(nvcc: str, src: str, obj: str, extra: list[str]) -> None:
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj + ".tmp"]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x=cu")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n"
                           f"{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)


def _link(nvcc: str, lib: str, objs: list[str], force: bool) -> None:
    if force or not os.path.exists(lib) or \
            os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False,
          extra_flags: list[str] | None = None, debug: bool = False) -> str:
    """Compile every CUDA translation unit, link libne.so and the probe's
    libne_probe.so; returns libne.so's path.  debug=True: link the
    index-checking libne_debug.so alone and return its path."""
    nvcc = _nvcc()
    bdir = BUILD_DEBUG if debug else BUILD
    os.makedirs(bdir, exist_ok=True)
    hdr = _headers_mtime()
    extra = list(extra_flags or []) + (["-DNE_INDEX_CHECKS"] if debug else [])
    jobs = []
    libs = ((DEBUG_LIB, SOURCES),) if debug else \
        ((LIB, SOURCES), (PROBE_LIB, PROBE_SOURCES))
    objs = {lib: [] for lib, _ in libs}
    for lib, names in libs:
        for name in names:
            src = os.path.join(CSRC, name)
            if not os.path.exists(src):
                continue
            obj = os.path.join(bdir, name + ".o")
            objs[lib].append(obj)
            if force or not os.path.exists(obj) or \
                    os.path.getmtime(obj) < max(os.path.getmtime(src), hdr):
                jobs.append((src, obj))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            futs = [ex.submit(_compile, nvcc, s, o, extra) for s, o in jobs]
            for f in futs:
                f.result()
    for lib, _ in libs:
        _link(nvcc, lib, objs[lib], force or bool(jobs))
    if verbose:
        print("built " + " and ".join(lib for lib, _ in libs))
    return libs[0][0]


if __name__ == "__main__":
    import sys
    build(verbose=True, debug="--debug" in sys.argv[1:])
