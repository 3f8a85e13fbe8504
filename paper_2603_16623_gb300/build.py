"""Builds libwake.so in-tree with nvcc for sm_103a.

    python -m paper_2603_16623_gb300.build [--bounds-check]

--bounds-check builds the debug library (_build_bc/libwake.so, compiled with
-DWAKE_BOUNDS_CHECK: the on-chip marches check every swizzled shared-memory
position and DSMEM peer rank, see wake_debug_bounds_violations); the
package loads it instead of the normal one when GBWAKE_BOUNDS_CHECK=1.

Each .cu file under csrc/ compiles to an object in parallel; the objects link
into paper_2603_16623_gb300/_build/libwake.so (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libwake.so")
BUILD_BC = os.path.join(HERE, "_build_bc")
LIB_BC = os.path.join(BUILD_BC, "libwake.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--cudart", "shared", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return exe


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def lib_for(bounds_check: bool = False) -> str:
    return LIB_BC if bounds_check else LIB


def up_to_date(bounds_check: bool = False) -> bool:
    lib = lib_for(bounds_check)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), bounds_check: bool = False) -> str:
    lib = lib_for(bounds_check)
    if not force and up_to_date(bounds_check):
        return lib
    bdir = os.path.dirname(lib)
    os.makedirs(bdir, exist_ok=True)
    srcs = _sources()
    objs = [os.path.join(bdir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    flags = [*FLAGS, *extra_flags] + (["-DWAKE_BOUNDS_CHECK"] if bounds_check else [])

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [nvcc(), *ARCH, *flags, "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
        if verbose:
            sys.stdout.write(res.stdout + res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, len(srcs))) as ex:
        list(ex.map(compile_one, zip(srcs, objs)))
    tmp = lib + f".{os.getpid()}.tmp"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc()))), "lib64")
    cmd = [nvcc(), *ARCH, "-shared", "--cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath", "-Xlinker", cuda_lib]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds_check="--bounds-check" in sys.argv))
