"""Build the CUDA library libeles.so (sm_103a) in-tree with nvcc.

Each translation unit under csrc/ is compiled in parallel, then linked into
paper_1902_02508_gb300/_lib/libeles.so.  No torch headers are involved: the
library exposes the plain C ABI of include/eles.h.
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
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libeles.so")
CHECK_DIR = os.path.join(HERE, "_lib_check")
CHECK_LIB = os.path.join(CHECK_DIR, "libeles_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
            "-I", INCLUDE, "-I", CSRC, *extra]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Build libeles.so; with check=True the range-checked debug library
    (-DELES_CHECK: every checked global index that falls outside its buffer
    records EF_ERR_RANGE in the error word and skips the access) in
    _lib_check/libeles_check.so, which eles.load() picks when the environment
    variable ELES_CHECK is 1."""
    out_dir, lib = (CHECK_DIR, CHECK_LIB) if check else (OUT_DIR, LIB)
    os.makedirs(out_dir, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
               + glob.glob(os.path.join(INCLUDE, "*.h")))
    objs = [os.path.join(out_dir, os.path.basename(s)[:-3] + ".o") for s in sources]
    todo = [(s, o) for s, o in zip(sources, objs) if force or _stale(o, [s, *headers])]

    def compile_one(so):
        s, o = so
        tmp = o + f".{os.getpid()}.tmp"   # per process: concurrent builds never share a file
        cmd = [nvcc(), *_flags(["-DELES_CHECK"] if check else []), "-c", s, "-o", tmp]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError(f"nvcc failed on {os.path.basename(s)}:\n{r.stderr}")
        os.replace(tmp, o)

    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            list(ex.map(compile_one, todo))
    if force or todo or _stale(lib, objs):
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
