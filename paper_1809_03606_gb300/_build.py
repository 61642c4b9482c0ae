"""Build libpolarscs.so in-tree with nvcc for sm_103a.

Translation units compile in parallel (one -gencode, no cmake); the shared
library lands in ``paper_1809_03606_gb300/_build/``.  Rebuilds only when a
source or header is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libpolarscs.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["plan.cpp", "api.cu", "scs_decode.cu", "encode.cu", "gsc.cu", "serve.cpp"]
# -fmad=false: the decoder's float arithmetic must not be contracted (bit
# parity with the CPU oracle): its only products, the optional stage scales,
# are rounded on their own before any sum.
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpolarscs")


def _deps() -> list[str]:
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return out


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def variant_lib(variant: str) -> str:
    return LIB if not variant else os.path.join(BUILD, f"libpolarscs_{variant}.so")


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, variant: str = "") -> str:
    """Build the library.  Variants are separate libraries for diagnosis:
    "timers" (libpolarscs_timers.so) with the per-phase cycle counters
    compiled in, "debug" (libpolarscs_debug.so) with the decoder's index
    checks (POLAR_DEBUG: a failed check marks the frame POLAR_DEBUG_FAIL)."""
    lib = variant_lib(variant)
    defines = {"": [], "timers": ["-DPOLAR_PHASE_TIMERS"], "debug": ["-DPOLAR_DEBUG"]}[variant]
    if not force and not needs_build(lib):
        return lib
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + (f".{variant}" if variant else "") + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *defines, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info and src.endswith(".cu"):
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0 or ptxas_info:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}")
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".{os.getpid()}.tmp"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc link of libpolarscs.so failed")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
