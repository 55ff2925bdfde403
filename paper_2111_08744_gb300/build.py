"""Build the CUDA library libmt.so in-tree for GB300 (sm_103a).

Each translation unit is compiled by nvcc in parallel (one -gencode, no cmake), then
linked into `paper_2111_08744_gb300/_build/libmt.so`.  Host code is compiled with
-ffp-contract=off so host-side arithmetic (eta_stop bisection) is plain IEEE.

FP64 forms are compiled without FMA contraction (`-fmad=false`), so every FP64 operation of
the double-precision path is one IEEE-754 operation, as in the method's definition:
  * a source whose first lines carry the marker `build: precision-split` is compiled twice,
    once as is (FP32-field instantiations and the entry points, contraction on) and once with
    -DMT_TU_FP64 -fmad=false (its FP64-field instantiations only);
  * a source marked `build: fp64` is compiled once, with -fmad=false.
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
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-Xptxas", "-O3",
              "-I", os.path.join(ROOT, "include")]
FP64_FLAGS = ["-DMT_TU_FP64", "-fmad=false"]


def nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmt.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _mode(src: str) -> str:
    """'split', 'fp64' or 'plain', from the marker in the source's first lines."""
    with open(src) as f:
        head = "".join(f.readline() for _ in range(5))
    if "build: precision-split" in head:
        return "split"
    if "build: fp64" in head:
        return "fp64"
    return "plain"


def _units():
    """(source, object, extra flags) for every translation unit."""
    units = []
    for s in _sources():
        stem = os.path.join(OUT, os.path.basename(s)[:-3])
        mode = _mode(s)
        if mode == "fp64":
            units.append((s, stem + ".o", FP64_FLAGS[1:]))
        else:
            units.append((s, stem + ".o", []))
        if mode == "split":
            units.append((s, stem + "_fp64.o", FP64_FLAGS))
    return units


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "mt.h"), __file__]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libmt.so if any source changed; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    units = _units()

    def compile_one(unit):
        src, obj, extra = unit
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(obj)}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(os.path.basename(obj), r.stderr)
        return obj

    # the slowest units first, so the parallel build ends soon after the longest one
    units.sort(key=lambda u: -os.path.getsize(u[0]))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(units), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *sorted(objs)], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
