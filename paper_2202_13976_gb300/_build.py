"""Compiles the CUDA library (sm_103a) into libtc.so inside the package directory.

nvcc compiles each translation unit in parallel with
``-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and links them with the
CUDA runtime into one shared library exporting the C ABI of include/tc.h.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libtc.so")
OBJDIR = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtc.so")
    return path


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs() -> list[str]:
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(ROOT, "include", "tc.h")]


# Source files that define the kernels of each measured phase: a DRAM-traffic record
# taken on them stays valid while these files are unchanged (the device headers hold
# the kernels' constants and helpers; include/tc.h only declares the C ABI).
KERNEL_SOURCES = {
    "hub": ["tc_intersect.cu", "tc_core.cu", "tc_device.cuh", "tc_internal.h"],
    "small": ["tc_intersect.cu", "tc_device.cuh", "tc_internal.h"],
    "directed": ["tc_directed.cu", "tc_device.cuh", "tc_internal.h"],
}


def source_digest(phase: str | None = None) -> str:
    """sha256 over the library sources, or over the files that define one measured
    phase's kernels (KERNEL_SOURCES): identifies the kernels a profile was taken on."""
    import hashlib
    h = hashlib.sha256()
    files = _inputs() if phase is None else [os.path.join(CSRC, f) for f in KERNEL_SOURCES[phase]]
    for p in sorted(files):
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    cc = nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(OBJDIR, os.path.basename(src).replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=PKG)
    os.close(fd)
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        os.unlink(tmp)
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB
