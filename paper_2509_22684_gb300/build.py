"""Build ``libzkntt.so`` in-tree with nvcc for sm_103a (no cmake, no torch
extension machinery): each translation unit compiles in parallel, then one
shared-library link.  Re-running skips units whose object is newer than every
source and header."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
# ZKNTT_NVCC_FLAGS adds compile flags (e.g. -DZKNTT_MUL_FORM=1) and
# ZKNTT_LIB_OUT names another output library, for building variants side by side
EXTRA = os.environ.get("ZKNTT_NVCC_FLAGS", "").split()
LIB = os.environ.get("ZKNTT_LIB_OUT") or os.path.join(HERE, "libzkntt.so")
OBJ = os.path.join(HERE, "_build") if LIB == os.path.join(HERE, "libzkntt.so") else LIB + ".objs"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}",
         "-Xptxas", "-warn-spills"]
UNITS = ["batch.cu", "kernels_bls12_381.cu", "kernels_bn254.cu", "kernels_bls12_377.cu", "zkntt.cu",
         "tuner.cu"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _headers_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(f) for f in files)


def _compile(unit: str, hdr_mtime: float, verbose: bool) -> str:
    src = os.path.join(CSRC, unit)
    obj = os.path.join(OBJ, unit.replace(".cu", ".o"))
    if os.path.exists(obj) and os.path.getmtime(obj) > max(os.path.getmtime(src), hdr_mtime):
        return obj
    cmd = [_nvcc(), *ARCH, *FLAGS, *EXTRA, "-c", src, "-o", obj + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{res.stdout}\n{res.stderr}")
    if res.stderr.strip() and verbose:
        print(res.stderr, file=sys.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OBJ, exist_ok=True)
    hdr = _headers_mtime()
    with cf.ThreadPoolExecutor(max_workers=jobs or len(UNITS)) as ex:
        objs = list(ex.map(lambda u: _compile(u, hdr, verbose), UNITS))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [_nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp", *objs]
        subprocess.run(cmd, check=True, capture_output=not verbose)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
