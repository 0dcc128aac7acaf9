"""Builds the CUDA library libdbar_gb300.so in-tree for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into one shared library with a plain C ABI (include/dbar.h).

    python -m paper_1508_02363_gb300.build
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libdbar_gb300.so")
SIZES = range(5, 12)  # N = 32 .. 2048
# (source, object name, extra flags): the pass kernels once per precision and size
UNITS = ([("kern_pass.cu", f"pass_{t}_{l}", [f"-DDBAR_T={t}", f"-DDBAR_LOGN={l}", f"-DDBAR_KIND={kind}"])
          for t, kind in (("double", 1), ("dd", 2), ("float", 0)) for l in SIZES] +
         [("kern_krylov.cu", "krylov", []), ("dispatch.cu", "dispatch", []), ("plan.cu", "plan", []),
          ("serve.cu", "serve", []), ("noalloc.cu", "noalloc", []), ("conv.cu", "conv", []),
          ("batches.cu", "batches", []),
          ("kern_aux.cu", "kern_aux", [])])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# extra nvcc flags (e.g. block-shape macros of csrc/cx.cuh) for tuning builds
EXTRA = os.environ.get("DBAR_NVCC_FLAGS", "").split()


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdbar_gb300.so")
    return exe


def _compile(unit, verbose: bool) -> str:
    src, name, flags = unit
    obj = os.path.join(BUILD, name + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *flags, *EXTRA,
           "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {name}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


STAMP = os.path.join(BUILD, "flags.txt")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    # a change of the extra flags (DBAR_NVCC_FLAGS) rebuilds everything
    if not os.path.exists(STAMP) or open(STAMP).read() != " ".join(EXTRA):
        return True
    t = os.path.getmtime(LIB)
    for f in os.listdir(CSRC):
        if os.path.getmtime(os.path.join(CSRC, f)) > t:
            return True
    return os.path.getmtime(os.path.join(ROOT, "include", "dbar.h")) > t


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    workers = max(1, min(len(UNITS), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(lambda u: _compile(u, verbose), UNITS))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(" ".join(EXTRA))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
