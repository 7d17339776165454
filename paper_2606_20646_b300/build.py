"""Build the sm_103a CUDA library ``liblbm_b300.so`` in-tree with nvcc."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "liblbm_b300.so")
# translation units and their extra flags: the FP64 unit is built without FMA contraction so that
# its arithmetic follows the FP64 oracle operation for operation
SOURCES = [(os.path.join(HERE, "csrc", "lbm_api.cu"), []),
           (os.path.join(HERE, "csrc", "lbm_fp32.cu"), []),
           (os.path.join(HERE, "csrc", "lbm_fp64.cu"), ["-fmad=false"]),
           (os.path.join(HERE, "csrc", "lbm_bf16s.cu"), []),
           (os.path.join(HERE, "csrc", "lbm_static.cu"), [])]
DEPENDS = glob.glob(os.path.join(HERE, "csrc", "*")) + [os.path.join(ROOT, "include", "lbm.h")]

NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-gencode", "arch=compute_103a,code=sm_103a",
              "-Xcompiler", "-fPIC"]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPENDS)


def build(force: bool = False, verbose: bool = False) -> str:
    if force or stale():
        objdir = os.path.join(HERE, "_build")
        os.makedirs(objdir, exist_ok=True)
        objs = []
        for src, extra in SOURCES:
            obj = os.path.join(objdir, os.path.basename(src).replace(".cu", ".o"))
            cmd = ["nvcc", *NVCC_FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-c", "-o", obj, src]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            subprocess.check_call(cmd)
            objs.append(obj)
        tmp = LIB + ".tmp"
        subprocess.check_call(["nvcc", "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
