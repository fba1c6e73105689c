"""Builds libfb.so in-tree with nvcc for sm_103a (B300)."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_PATH = os.path.join(PKG, "libfb.so")
SOURCES = ["fb_api.cu", "fb_kernels.cu", "fb_batch.cu", "fb_net.cu", "fb_calib.cu", "fb_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    files.append(os.path.join(INCLUDE, "fb.h"))
    return files


def is_stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(f) > t for f in _inputs())


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


DEBUG_LIB_PATH = os.path.join(PKG, "libfb_debug.so")


def _compile(out: str, defines=(), verbose: bool = False, ptxas_info: bool = False) -> str:
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-shared", "-I", INCLUDE, "-I", CSRC, "-o", tmp]
    cmd += [f"-D{d}" for d in defines]
    if ptxas_info:
        cmd += ["-Xptxas", "-v"]
    cmd += [os.path.join(CSRC, s) for s in SOURCES]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _stale(path: str) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every CUDA source of the package into libfb.so (skip if up to date)."""
    if not force and not is_stale():
        return LIB_PATH
    return _compile(LIB_PATH, verbose=verbose, ptxas_info=ptxas_info)


def build_debug(force: bool = False, verbose: bool = False) -> str:
    """libfb_debug.so: the same sources with FB_COUNT_EVALS (candidate counter)."""
    if not force and not _stale(DEBUG_LIB_PATH):
        return DEBUG_LIB_PATH
    return _compile(DEBUG_LIB_PATH, defines=("FB_COUNT_EVALS",), verbose=verbose)


CHECKED_LIB_PATH = os.path.join(PKG, "libfb_checked.so")


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """libfb_checked.so: the same sources with FB_CHECKED (device-side invariant checks
    that record failures in a status word instead of faulting; fb_check_status)."""
    if not force and not _stale(CHECKED_LIB_PATH):
        return CHECKED_LIB_PATH
    return _compile(CHECKED_LIB_PATH, defines=("FB_CHECKED",), verbose=verbose)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB_PATH)
