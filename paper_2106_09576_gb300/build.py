"""Builds libdem_gb300.so (the CUDA library behind include/dem.h and include/surrogate.h)
in-tree for sm_103a.

The translation units are compiled in parallel with nvcc, then linked as one shared
library in paper_2106_09576_gb300/_build/.  The FP64 step kernel is compiled without
FMA contraction so that it rounds like the serial CPU statement of the method.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libdem_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = {
    "dem_api.cu": [],
    "dem_rebuild.cu": [],
    "dem_step_fp64.cu": ["-fmad=false"],
    # FP32 division and square root need not be correctly rounded in the mixed kernel;
    # additions, multiplications and FMAs stay IEEE (the double-float arithmetic needs them)
    "dem_step_mixed.cu": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"],
    "dem_static_pairs.cu": [],
    "dem_probe.cu": [],
    "surrogate.cu": [],
    "surrogate_tc.cu": [],
}


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdem_gb300.so")


def _inputs():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "dem.h"))
    deps.append(os.path.join(ROOT, "include", "surrogate.h"))
    deps.append(os.path.abspath(__file__))
    return deps


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nv = nvcc()
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                     "-I", os.path.join(ROOT, "include")]

    def compile_one(item):
        src, extra = item
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [nv] + common + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES.items()))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nv] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
