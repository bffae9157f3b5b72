"""Builds libpsfs.so in-tree with nvcc for sm_103a (GB300).

The translation units compile in parallel to objects, then link into one
shared library with the CUDA runtime linked statically.  The library has a
plain C ABI (include/psfs.h); no torch types cross it.
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
LIB = os.path.join(BUILD, "libpsfs.so")
# the bounds-checked build (-DPSFS_BOUNDS_CHECK): device-side index checks at
# the gathers and stores whose indices rest on the kernels' own arithmetic or
# on the planner's proofs; a failed check skips the access and psfs_sync
# returns PSFS_ERR_BOUNDS.  For tests; the product build is LIB.
BOUNDS_BUILD = os.path.join(HERE, "_build_bounds")
BOUNDS_LIB = os.path.join(BOUNDS_BUILD, "libpsfs.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpsfs")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), bounds_check: bool = False) -> str:
    """Compiles the sources that changed and links the library; returns its
    path (LIB, or BOUNDS_LIB with `bounds_check`)."""
    build_dir, lib = (BOUNDS_BUILD, BOUNDS_LIB) if bounds_check else (BUILD, LIB)
    if bounds_check:
        extra_flags = (*extra_flags, "-DPSFS_BOUNDS_CHECK")
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "psfs.h"))
    srcs = sources()
    objs = [os.path.join(build_dir, os.path.basename(s).replace(".cu", ".o")) for s in srcs]
    nv = nvcc()
    jobs = []
    for s, o in zip(srcs, objs):
        if force or _stale(o, [s] + headers):
            jobs.append([nv, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", s, "-o", o])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, res in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
            if verbose or res.returncode != 0:
                print(" ".join(cmd))
                print(res.stdout, res.stderr)
            if res.returncode != 0:
                raise RuntimeError(f"nvcc failed on {cmd[-3]}")
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            print(" ".join(cmd))
            print(res.stdout, res.stderr)
            raise RuntimeError("link of libpsfs.so failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
