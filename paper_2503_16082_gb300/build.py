"""Build libsphst.so in-tree with nvcc for sm_103a (one -gencode, the three
translation units compiled in parallel)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsphst.so")
SOURCES = ["sphst_api.cu", "sphst_f32.cu", "sphst_f64.cu", "sphst_noalloc.cu", "sphst_peak.cu"]
HEADERS = ["sphst_internal.cuh", "sphst_kernels.cuh", "sphst_engine.cuh", "sphst_engine_impl.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-I", os.path.join(HERE, "..", "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link; SPHST_NVCC_DEFINES (e.g. "-DSPHST_SWEEP_MINB=4")
    adds tuning defines.  The defines of the last build are recorded, and a
    change of them rebuilds everything."""
    os.makedirs(BUILD, exist_ok=True)
    extra = os.environ.get("SPHST_NVCC_DEFINES", "").split()
    stamp = os.path.join(BUILD, "defines.txt")
    recorded = open(stamp).read() if os.path.exists(stamp) else None
    if recorded != " ".join(extra):
        force = True
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "sphst.h")]
    objs = []
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            jobs.append([nvcc(), *FLAGS, *extra, *ARCH, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(" ".join(extra))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
