"""Build the CUDA library in-tree for sm_103a with nvcc (no cmake).

Each translation unit is compiled in parallel, then linked into
``paper_2409_02930_gb300/_build/liblbm.so``.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include")]


def per_file_flags(src):
    """The FP32 kernel units use the fast (few-ulp) division, square root and
    power; their FP32 results are compared with the FP64 oracle at 1e-5.
    The FP64 units keep IEEE division and square root."""
    return ["--use_fast_math"] if "_f32_" in os.path.basename(src) else []


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(ROOT, "include", "lbm.h"))
    return hs


def _deps(depfile, fallback):
    """Headers a unit includes, from the dependency file of its last build
    (every header when there is none)."""
    try:
        with open(depfile) as f:
            text = f.read().replace("\\\n", " ")
    except OSError:
        return fallback
    _, _, rest = text.partition(":")
    files = [t for t in rest.split() if t.endswith((".cuh", ".h"))]
    files = [f for f in files if os.path.abspath(f).startswith(ROOT)]
    return files or fallback


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    hdrs = _headers()
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        dep = obj[:-2] + ".d"
        objs.append(obj)
        if force or _stale(obj, [src] + _deps(dep, hdrs)):
            cmd = [nvcc, "-c", src, "-o", obj, "-MD", "-MF", dep] + ARCH + FLAGS + per_file_flags(src) + list(extra)
            jobs.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr

    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for out in ex.map(run, jobs):
                if verbose and out:
                    print(out, file=sys.stderr)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
