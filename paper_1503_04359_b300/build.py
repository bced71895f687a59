"""Builds libdobfs.so (the C-ABI library) from csrc/*.cu for sm_103a.

    python -m paper_1503_04359_b300.build [--force] [--verbose] [--bounds-check]

With --bounds-check the same sources are compiled with -DDOBFS_BOUNDS_CHECK
into ``_lib/libdobfs_bc.so``: every index the kernels read from memory is
checked on the device and a failure is reported as DOBFS_ERR_BOUNDS (the
binding loads this variant when DOBFS_BOUNDS_CHECK=1 is set).

Every .cu is compiled to an object with nvcc (in parallel) and linked into
``_lib/libdobfs.so`` with the shared CUDA runtime, so the library shares the
runtime PyTorch already loaded when both live in one process.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
REPO = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
BUILD_DIR = os.path.join(REPO, "_build", "dobfs")
LIB = os.path.join(OUT_DIR, "libdobfs.so")
LIB_BC = os.path.join(OUT_DIR, "libdobfs_bc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                     "--expt-relaxed-constexpr", "-I" + os.path.join(REPO, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _deps() -> list[str]:
    files = []
    for d in (CSRC, os.path.join(REPO, "include"), os.path.join(REPO, "dobfs_inputs")):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")):
                files.append(os.path.join(d, f))
    return files


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          bounds_check: bool = False) -> str:
    """Compile (if stale) and return the path of libdobfs.so (libdobfs_bc.so
    with bounds_check)."""
    lib = LIB_BC if bounds_check else LIB
    build_dir = BUILD_DIR + ("_bc" if bounds_check else "")
    newest = max(os.path.getmtime(f) for f in _deps() + [__file__])
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest and not extra_flags:
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    flags = NVCC_FLAGS + (["-DDOBFS_BOUNDS_CHECK"] if bounds_check else []) + (extra_flags or [])

    def compile_one(src: str) -> str:
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
        "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else None
    print(build(force="--force" in sys.argv or extra is not None, verbose="--verbose" in sys.argv or extra is not None,
                extra_flags=extra, bounds_check="--bounds-check" in sys.argv))
