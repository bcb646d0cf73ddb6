"""Build the SGF CUDA library in-tree (nvcc for sm_103a, no cmake).

Produces paper_1907_03406_gb300/lib/libsgf.so from csrc/: the device kernels
(kernels.cu) and the host runtime (analysis, factor driver, C ABI).  The
translation units compile in parallel; the CUDA runtime is linked statically.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "lib")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _sources():
    return sorted(f for f in os.listdir(SRC) if f.endswith((".cu", ".cpp")))


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    os.makedirs(BUILD, exist_ok=True)
    lib = os.path.join(OUT, "libsgf.so")
    srcs = _sources()
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(ROOT, "include", "sgf.h")]
    if not force and os.path.exists(lib):
        newest = max(os.path.getmtime(d) for d in deps)
        if os.path.getmtime(lib) >= newest:
            return lib
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", SRC]
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo"] + inc

    def compile_one(f):
        obj = os.path.join(BUILD, f + ".o")
        if f.endswith(".cu"):
            cmd = [nvcc] + ARCH + common + ["--expt-relaxed-constexpr", "-c", os.path.join(SRC, f), "-o", obj]
        else:
            cmd = [nvcc] + common + ["-x", "cu", "-c", os.path.join(SRC, f), "-o", obj] + ARCH
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {f}\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
