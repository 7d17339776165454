"""Build the sm_103a CUDA library in-tree with nvcc: ``liblbm_b300.so`` and its bounds-checked
twin ``liblbm_b300_check.so`` (-DLBM_CHECK: data-dependent indices checked in the kernels, a
violation latched as LBM_DEV_BOUNDS)."""
from __future__ import annotations

import fcntl
import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "liblbm_b300.so")
LIB_CHECK = os.path.join(HERE, "liblbm_b300_check.so")
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


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in DEPENDS)


def _link(lib: str, objdir: str, extra: list, verbose: bool) -> list:
    """nvcc commands of one library: the objects, then the shared-object link."""
    os.makedirs(objdir, exist_ok=True)
    compiles, objs = [], []
    for src, flags in SOURCES:
        obj = os.path.join(objdir, os.path.basename(src).replace(".cu", ".o"))
        cmd = ["nvcc", *NVCC_FLAGS, *flags, *extra, "-I", os.path.join(ROOT, "include"), "-c", "-o", obj, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        compiles.append(cmd)
        objs.append(obj)
    link = ["nvcc", "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", lib + ".tmp", *objs]
    return compiles, link


def build(force: bool = False, verbose: bool = False, check: bool = True) -> str:
    """Compile both libraries (the checked one unless check=False) when a source is newer; the
    translation units compile in parallel.  Callers in several processes (one per rank) take turns
    on a lock file, so one compiles and the others then find the libraries current."""
    os.makedirs(os.path.join(HERE, "_build"), exist_ok=True)
    with open(os.path.join(HERE, "_build", ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            return _build_locked(force, verbose, check)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(force: bool, verbose: bool, check: bool) -> str:
    targets = [(LIB, os.path.join(HERE, "_build"), [])]
    if check:
        targets.append((LIB_CHECK, os.path.join(HERE, "_build_check"), ["-DLBM_CHECK"]))
    todo = [t for t in targets if force or stale(t[0])]
    if todo:
        jobs, links = [], []
        for lib, objdir, extra in todo:
            c, l = _link(lib, objdir, extra, verbose)
            jobs += c
            links.append((lib, l))
        with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
            for f in [ex.submit(subprocess.check_call, cmd) for cmd in jobs]:
                f.result()
        for lib, l in links:
            subprocess.check_call(l)
            os.replace(lib + ".tmp", lib)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
