"""Build and load the native library (libgwn.so) of the GWN package.

The library is compiled in-tree with nvcc for sm_103a (GB300) from the sources
under csrc/; host translation units go through g++.  Nothing here falls back
to Python: if the library cannot be built or loaded, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libgwn.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["gwn_api.cu", "gwn_serve.cu", "gwn_batch.cu", "build_device.cu"]
# the device stage of the build must round like the host stage: no fused multiply-adds
CU_FLAGS = {"build_device.cu": ["-fmad=false"]}
CPP_SOURCES = ["build.cpp", "build3d.cpp"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgwn.so")


def _sources():
    cu = [s for s in CU_SOURCES if os.path.exists(os.path.join(CSRC, s))]
    return cu, CPP_SOURCES


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "gwn.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.isfile(d))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libgwn.so in-tree (parallel translation units).  Returns its path."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    cu, cpp = _sources()
    jobs = []
    for s in cu:
        o = os.path.join(BUILD_DIR, s + ".o")
        jobs.append([nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, *CU_FLAGS.get(s, []), "-Xcompiler", "-fPIC",
                     "-I", INCLUDE, "-c", os.path.join(CSRC, s), "-o", o])
    for s in cpp:
        o = os.path.join(BUILD_DIR, s + ".o")
        # no contraction into fused multiply-adds (g++ contracts by default on
        # aarch64): the host stage of the 3D build must round like the device stage
        jobs.append(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-I", INCLUDE, "-I", CSRC, "-pthread",
                     "-c", os.path.join(CSRC, s), "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            print(r.stdout + r.stderr)
        return cmd[-1]

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(run, jobs))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    link = [nvcc, "-shared", *ARCH, "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + " ".join(link) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def load() -> ctypes.CDLL:
    """Load libgwn.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = build()
        _lib = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
    return _lib
