"""Compile the CUDA library ``libdgw.so`` in-tree for sm_103a with nvcc.

Each translation unit is compiled in its own nvcc process (in parallel), then
linked into one shared library next to this file.  The CUDA runtime is linked
statically, so the library has no dependency on a particular libcudart.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdgw.so")
LIB_DEBUG = os.path.join(HERE, "libdgw_debug.so")
SOURCES = ["dgw_capi.cu", "dgw_batch.cu", "dgw_adjoint.cu", "dgw_geometry.cu", "dgw_energy.cu", "dgw_energy_static.cu", "dgw_stage_fp64.cu",
           "dgw_stage_mixed.cu", "dgw_stage_mixed_tc.cu", "dgw_friedrichs.cu", "dgw_ihdg.cu", "dgw_probe.cu", "dgw_state.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdgw.so")
    return path


def _inputs_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "dgw.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    """Build (if stale) and return the path of libdgw.so, or with debug=True of
    libdgw_debug.so (device-side checks, -DDGW_DEBUG_CHECKS)."""
    lib = LIB_DEBUG if debug else LIB
    bdir = BUILD + "_debug" if debug else BUILD
    flags = [*extra_flags, "-DDGW_DEBUG_CHECKS"] if debug else list(extra_flags)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _inputs_mtime():
        return lib
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
