"""In-tree build of the CUDA library ``_lib/libpf_gb300.so`` for sm_103a.

Three translation units are compiled in parallel with nvcc and linked into one shared
library: the FP32 kernels, the FP64 kernels (no fused multiply-add contraction, so their
rounding follows the written expressions) and the host runtime behind the C ABI.
Host code is compiled with -ffp-contract=off so that host arithmetic (the default time
step, the Voronoi seeds) rounds the same on x86-64 and aarch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libpf_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", f"-I{INCLUDE}"]

# The FP32 unit takes the hardware's approximate single-precision division and square root (within
# 2 ulp; the anti-trapping current's normals and weights divide and take roots on every interface
# face): the general planes' sweeps run 17 % faster, and the FP32 results stay within their stated
# tolerance of the FP64 oracle.  The FP64 unit keeps IEEE operations without contraction.
UNITS = {
    "pf_kernels_f32.cu": ["-prec-div=false", "-prec-sqrt=false"],
    "pf_kernels_f64.cu": ["-fmad=false"],
    "pf_api.cpp": [],
    "pf_noalloc.cu": [],
}


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpf_gb300.so")


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".cpp", ".h"))]
    deps.append(os.path.join(INCLUDE, "pf.h"))
    deps.append(os.path.abspath(__file__))
    return deps


def is_stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not is_stale():
        return LIB
    nvcc = _nvcc()
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)

    def compile_unit(name):
        src = os.path.join(CSRC, name)
        obj = os.path.join(obj_dir, name + ".o")
        cmd = [nvcc, *ARCH, *COMMON, *UNITS[name], "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=False))
