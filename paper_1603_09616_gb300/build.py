"""Build the in-tree CUDA library ``libgbgreen.so`` for sm_103a (GB300).

Three translation units: ``csrc/solver.cu`` (solver kernels + C ABI),
``csrc/surrogate.cu`` (descriptor and MLP kernels) and ``csrc/bsr_build.cpp``
(host CSR -> 4x4 block builder), compiled in parallel and linked with nvcc
into ``paper_1603_09616_gb300/libgbgreen.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgbgreen.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbgreen.so")
    return cand


def build_library(force: bool = False, verbose: bool = False) -> str:
    srcs = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    nvcc = _nvcc()
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    obj_cu = os.path.join(bdir, "solver.o")
    obj_sg = os.path.join(bdir, "surrogate.o")
    obj_cpp = os.path.join(bdir, "bsr_build.o")
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC"]
    cmds = [
        [nvcc, ARCH, "-lineinfo", *common, "-c", os.path.join(CSRC, "solver.cu"), "-o", obj_cu],
        [nvcc, ARCH, "-lineinfo", *common, "-c", os.path.join(CSRC, "surrogate.cu"), "-o", obj_sg],
        [nvcc, *common, "-c", os.path.join(CSRC, "bsr_build.cpp"), "-o", obj_cpp],
    ]
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if p.returncode != 0:
            raise RuntimeError(f"build step failed: {' '.join(c)}\n{out}")
    tmp = LIB + ".tmp"
    link = [nvcc, ARCH, "-shared", "-o", tmp, obj_cu, obj_sg, obj_cpp, "-lcudart"]
    res = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{res.stdout}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True))
