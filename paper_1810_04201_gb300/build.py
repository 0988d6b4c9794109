"""Build libwd.so (the CUDA library) in-tree for sm_103a with nvcc.

Each translation unit under ``csrc/`` is compiled in parallel; the objects are
linked into ``paper_1810_04201_gb300/_build/libwd.so`` together with the static
CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD_RELEASE = os.path.join(HERE, "_build")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB = os.path.join(BUILD_RELEASE, "libwd.so")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libwd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwd")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra_flags=None, jobs: int | None = None, debug: bool = False) -> str:
    """Compile (what is stale) and link; debug=True builds the index-checking variant
    (-DWD_DEBUG) into _build_debug/libwd.so instead."""
    BUILD = BUILD_DEBUG if debug else BUILD_RELEASE
    LIB = os.path.join(BUILD, "libwd.so")
    if debug:
        extra_flags = list(extra_flags or []) + ["-DWD_DEBUG"]
    os.makedirs(BUILD, exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(os.path.dirname(HERE), "include", "wd.h")]
    srcs = sources()
    objs = []
    todo = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if _stale(o, [s] + headers):
            cmd = [nvcc()] + ARCH + NVCC_FLAGS + list(extra_flags or []) + ["-c", s, "-o", o]
            todo.append(cmd)
    jobs = jobs or min(len(todo), os.cpu_count() or 4) or 1

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for cmd, r in ex.map(run, todo):
            if verbose or r.returncode != 0:
                print(" ".join(cmd))
                print(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    if _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            print(r.stdout + r.stderr)
            raise RuntimeError("linking libwd.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv))
