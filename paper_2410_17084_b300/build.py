"""Build the sm_103a shared library of the Voxel-GPR path with nvcc (in-tree).

Each .cu file is compiled to its own object (in parallel, and only when it or a header
changed), then the objects are linked into libgp_voxels.so.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgp_voxels.so")
SOURCES = ["gpv_api.cu", "gpv_solve.cu", "gpv_store.cu", "gpv_noalloc.cu", "gpv_alg3.cu",
           "gpv_lp.cu", "gpv_raster.cu", "gpv_peak.cu", "gpv_vartc.cu", "gpv_tall.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
         "-fvisibility=hidden", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    c = "/usr/local/cuda/bin/nvcc"
    return c if os.path.exists(c) else "nvcc"


def _includes(path: str, seen: set[str] | None = None) -> set[str]:
    """Local headers a source includes, directly or through other headers."""
    seen = set() if seen is None else seen
    d = os.path.dirname(path)
    with open(path) as f:
        for line in f:
            t = line.strip()
            if t.startswith("#include \""):
                h = os.path.normpath(os.path.join(d, t.split('"')[1]))
                if os.path.exists(h) and h not in seen:
                    seen.add(h)
                    _includes(h, seen)
    return seen


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    objs, todo = [], []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OBJ, s[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src, *_includes(src), __file__]):
            cmd = [nvcc(), *ARCH, *FLAGS, "-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            todo.append(cmd)
    if todo:
        with ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            rcs = list(ex.map(lambda c: subprocess.call(c), todo))
        if any(rcs):
            raise subprocess.CalledProcessError(max(rcs), "nvcc")
    if todo or _stale(LIB, objs):
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"])
    return LIB


if __name__ == "__main__":
    build(force="-f" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
