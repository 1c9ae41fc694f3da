"""Build the in-tree CUDA library libnsfr.so for sm_103a (nvcc, no cmake).

Every translation unit is compiled in parallel with
  nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo -O3 -Xcompiler -fPIC
and linked into ``paper_2312_07725_gb300/libnsfr.so``.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnsfr.so")
SOURCES = ["api.cu", "ops1d.cpp", "geometry.cu", "residual.cu", "residual_bulk.cu", "reduce.cu", "vjp.cu", "mathfn.cu", "projection.cu", "source.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _compile(src, verbose_ptxas=False):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17", "-lineinfo",
           "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC] + ARCH
    # extra definitions for measuring a variant, e.g. NSFR_NVCC_DEFINES="-DNSFR_VOL_STAGE_TMA=0"
    cmd += [f for f in os.environ.get("NSFR_NVCC_DEFINES", "").split() if f.startswith("-D")]
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(verbose_ptxas=False, quiet=True):
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    objs = [o for o, _ in results]
    if verbose_ptxas:
        for (_, log), src in zip(results, SOURCES):
            print(f"== {src}\n{log}", file=sys.stderr)
    cmd = [nvcc(), "-shared", "-o", LIB] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    if not quiet:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(verbose_ptxas="-v" in sys.argv, quiet=False)
