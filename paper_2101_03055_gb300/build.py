"""Build libcdflb.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel; the shared library is linked
only when a source or header is newer than it.  No CMake, no torch extension
machinery: the library is plain C ABI and loads with ctypes.

build(checks=True) builds the checks library libcdflb_checks.so instead (the
same sources with -DCDF_CHECKS: offset checks in the step kernels, canary pads
around device buffers; see include/cdf_lb.h), which the binding loads when the
environment sets CDF_CHECKS=1.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcdflb.so")
LIB_CHECKS = os.path.join(PKG, "libcdflb_checks.so")
HEADERS = [os.path.join(ROOT, "include", "cdf_lb.h"), os.path.join(ROOT, "include", "cdf_lb3d.h"),
           os.path.join(ROOT, "include", "cdf_nn.h"), os.path.join(CSRC, "lb_internal.h"), os.path.join(CSRC, "lb_device.cuh")]
SOURCES = ["lb_kernels.cu", "lb_reduce.cu", "lb_host.cu", "lb_static.cu", "lb_batch.cu", "lb_resident.cu", "lb_split.cu",
           "lb_checks.cu", "lb3d.cu", "nn_kernels.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcdflb")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra, objdir: str = OBJ) -> str:
    obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    if _stale(obj, [path] + HEADERS):
        cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", path, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, extra=(), checks: bool = False) -> str:
    objdir, lib = (OBJ + "_checks", LIB_CHECKS) if checks else (OBJ, LIB)
    flags = list(extra) + (["-DCDF_CHECKS"] if checks else [])
    os.makedirs(objdir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, flags, objdir), SOURCES))
    if _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}")
    return lib


def ptxas_report() -> str:
    """Register / spill / shared-memory report of the step kernels (-Xptxas -v)."""
    out = []
    for src in SOURCES:
        cmd = [nvcc(), *ARCH, *FLAGS, "-Xptxas", "-v", "-c", os.path.join(CSRC, src), "-o", os.devnull]
        r = subprocess.run(cmd, capture_output=True, text=True)
        out.append(r.stderr)
    return "\n".join(out)


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "--ptxas":
        print(ptxas_report())
    else:
        build(verbose=True)
