"""Build libifem.so (the CUDA kernels behind include/ifem.h) for sm_103a.

Four translation units are compiled in parallel with nvcc and linked into
``paper_1807_08219_gb300/_build/libifem.so``:
  api.cu          host code (handles, checks, FP64 reference data), host
                  compiler with -ffp-contract=off
  kernels_f32.cu  FP32 kernels (FMA contraction allowed)
  kernels_f64.cu  FP64 deterministic kernels, --fmad=false
  noalloc.cu      the allocation-free force entry point, --fmad=false
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libifem.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {
    "api.cu": [],
    "kernels_f32.cu": [],
    "kernels_f64.cu": ["--fmad=false"],
    "noalloc.cu": ["--fmad=false"],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libifem")


def _sources_mtime() -> float:
    ts = [os.path.getmtime(os.path.join(CSRC, f)) for f in os.listdir(CSRC)]
    ts.append(os.path.getmtime(os.path.join(INCLUDE, "ifem.h")))
    ts.append(os.path.getmtime(__file__))
    return max(ts)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile libifem.so if it is missing or older than its sources."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "-I", INCLUDE, "-I", CSRC] + ARCH + (extra or [])
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(name: str) -> str:
        obj = os.path.join(BUILD, name.replace(".cu", ".o"))
        cmd = [cc, "-c", os.path.join(CSRC, name), "-o", obj] + common + UNITS[name]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {name}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, "-shared", "-o", tmp] + objs + ["-cudart", "shared"] + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
