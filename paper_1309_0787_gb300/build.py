"""Build the CUDA library ``_build/libotm.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` translation unit is compiled in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a``), then linked into one shared
library with the CUDA runtime.  Rebuilds only what changed (source newer than
its object).  Usage: ``python -m paper_1309_0787_gb300.build [-v]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libotm.so")
HEADERS = [os.path.join(SRC, f) for f in sorted(os.listdir(SRC)) if f.endswith(".cuh")] + [
    os.path.join(os.path.dirname(HERE), "include", "otm.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libotm")


def _stale(src: str, obj: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + HEADERS)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    # objects built on another host architecture (x86_64 vs aarch64) are rebuilt
    stamp = os.path.join(OUT, "HOST_ARCH")
    host = platform.machine()
    if force or not os.path.exists(stamp) or open(stamp).read().strip() != host:
        for f in os.listdir(OUT):
            if f.endswith((".o", ".so")):
                os.remove(os.path.join(OUT, f))
        with open(stamp, "w") as fh:
            fh.write(host + "\n")
    sources = sorted(f for f in os.listdir(SRC) if f.endswith(".cu"))
    jobs = []
    for f in sources:
        src = os.path.join(SRC, f)
        obj = os.path.join(OUT, f[:-3] + ".o")
        if _stale(src, obj):
            jobs.append([nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {cmd[-3]}:\n{res.stdout}\n{res.stderr}")
        return res

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(OUT, f[:-3] + ".o") for f in sources]
    if jobs or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB)
                                              for o in objs):
        run([nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-lcudart",
             "-Xlinker", "-rpath,/usr/local/cuda/lib64"])
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
