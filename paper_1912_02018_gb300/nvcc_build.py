"""Build liblbm.so (the C-ABI CUDA library) in-tree for sm_103a with nvcc.

Translation units, compiled in parallel:
  lbm_f64.cu  FP64 kernels, --fmad=false (products and sums rounded as written)
  lbm_f32.cu  FP32 kernels, FMA contraction allowed
  lbm_api.cu  host side of the C ABI (-ffp-contract=off so host FP64 thermodynamics
              round the same on x86-64 and aarch64)
  lbm_noalloc.cu  the allocation-free wall heat flux
  lbm_adjoint_api.cu  host side of the adjoint window (the FP32 reverse kernels sit in lbm_f32.cu)
  lbm_adjoint_f64.cu  FP64 reverse kernels of the adjoint, FMA contraction allowed
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
                 f"-I{INCLUDE}", f"-I{CSRC}"]
UNITS = {
    "lbm_f64.cu": ["--fmad=false"],
    "lbm_f32.cu": ["--fmad=true"],
    "lbm_api.cu": [],
    "lbm_noalloc.cu": [],
    "lbm_adjoint_api.cu": [],
    "lbm_adjoint_f64.cu": ["--fmad=true"],
}


def _sources_newer(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lbm.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _sources_newer(LIB):
        return LIB
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(name):
        obj = os.path.join(BUILD, name.replace(".cu", ".o"))
        cmd = [NVCC] + COMMON + UNITS[name] + ["-c", os.path.join(CSRC, name), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
        "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
