"""Builds libdg.so in-tree (``paper_2205_11638_gb300/_build/``) with nvcc for
sm_103a.  Translation units compile in parallel; nothing is installed."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libdg.so")
ROOT = os.path.dirname(HERE)

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc") if os.path.exists(os.path.join(CUDA_HOME, "bin", "nvcc")) else "nvcc"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                   f"-I{os.path.join(ROOT, 'include')}"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-pthread", f"-I{os.path.join(CUDA_HOME, 'include')}",
             f"-I{os.path.join(ROOT, 'include')}"]

SOURCES = ["builder.cpp", "api.cu", "kernels_sweep.cu", "kernels_misc.cu", "kernels_adjoint.cu", "kernels_long.cu",
           "kernels_params.cu", "noalloc.cu"]
HEADERS = ["dg_internal.h", "kernels.h", "sweep.cuh"]


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, extra=()):
    path = os.path.join(CSRC, src)
    obj = os.path.join(OUT, src + ".o")
    deps = [path] + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "dg.h")]
    if not _stale(obj, deps):
        return obj
    if src.endswith(".cpp"):
        cmd = ["g++", *CXX_FLAGS, "-c", path, "-o", obj + ".tmp"]
    else:
        cmd = [NVCC, *CU_FLAGS, *extra, "-c", path, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if force:
        for f in os.listdir(OUT):
            os.remove(os.path.join(OUT, f))
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    if _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
