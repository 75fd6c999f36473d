"""Build the in-tree CUDA library ``libcetra.so`` for sm_103a (nvcc + g++, no cmake).

The translation units compiled in parallel and linked into one shared
library next to this file:
  csrc/kernels.cu  resample, linear, finalize and batch kernels (nvcc, sm_103a)
  csrc/fold.cu     the single-curve fold kernel and its launcher (nvcc, sm_103a)
  csrc/fold_batch.cu  the batched fold kernel and its launcher (nvcc, sm_103a); both fold
                   files include the shared device code of csrc/fold.cuh
  csrc/plan.cpp    host planner, FP64 index arithmetic  (g++, -ffp-contract=off)
  csrc/capi.cpp    the C ABI declared in include/cetra.h (g++)
  csrc/noalloc.cu  the allocation-free periodic entry point (nvcc)
  csrc/batch.cpp   the batched form: layout, CUDA graph, autotuner (g++)
  csrc/cnn.cu      the learned period-interval proposal: CNN kernels and comb (nvcc)
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "libcetra.so")
BUILD = os.path.join(HERE, "_build")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES = ["kernels.cu", "fold.cu", "fold_batch.cu", "plan.cpp", "capi.cpp", "noalloc.cu", "batch.cpp", "cnn.cu",
           "neighbours.cu"]


def _cmd(src: str, obj: str) -> list[str]:
    path = os.path.join(CSRC, src)
    if src.endswith(".cu"):
        return [NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC, "-c", path, "-o", obj]
    return ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", "-I", INCLUDE,
            "-I", CSRC, "-I", os.path.join(CUDA, "include"), "-c", path, "-o", obj]


def _stale() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "cetra.h"),
                                                                  os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of libcetra.so."""
    if not force and not _stale():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        cmd = _cmd(src, obj)
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append(f"{src}:\n{out.decode(errors='replace')}")
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        raise RuntimeError("CUDA library build failed:\n" + "\n".join(failed))
    tmp = OUT + ".tmp"
    link = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    subprocess.run(link, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
