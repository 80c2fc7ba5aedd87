"""Build libnyxrt.so in-tree for sm_103a (GB300).

Each translation unit is compiled in its own process (in parallel), then
linked with nvcc. Host code is compiled with -ffp-contract=off so that the
host-side constants (split radius, cell size, direction table) are the plain
IEEE evaluation of their formulas.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libnyxrt.so")
PROBE_LIB = os.path.join(HERE, "libnyxrt_probe.so")   # arithmetic-peak probe, beside the library
BUILD = os.path.join(ROOT, "_build", "nyxrt")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SOURCES = ["march.cu", "fields.cu", "sources.cu", "rt_api.cu", "batch.cu", "server.cu", "noalloc.cu"]
CXX_SOURCES = ["directions.cpp"]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnyxrt")


def _cuda_home() -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(_nvcc())))


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "nyxrt.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    path = os.path.join(CSRC, src)
    if src.endswith(".cu"):
        cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-I", INCLUDE,
               "-Xcompiler", "-fPIC,-ffp-contract=off", "-c", path, "-o", obj]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I", INCLUDE,
               "-I", os.path.join(_cuda_home(), "include"), "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build_probe(force: bool = False) -> str:
    """The FMA-throughput probe (probe_peaks.cu) as its own shared library."""
    src = os.path.join(CSRC, "probe_peaks.cu")
    if not force and os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= os.path.getmtime(src):
        return PROBE_LIB
    tmp = PROBE_LIB + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", src, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    build_probe(force)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(CUDA_SOURCES) + len(CXX_SOURCES)) as ex:
        objs = list(ex.map(_compile, CUDA_SOURCES + CXX_SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


def ptxas_report(src: str = "march.cu") -> str:
    """Registers / spills / shared memory per kernel (nvcc -Xptxas -v)."""
    cmd = [_nvcc(), *ARCH, "-O3", "-std=c++17", "-I", INCLUDE, "-Xptxas", "-v", "-Xcompiler", "-fPIC",
           "-c", os.path.join(CSRC, src), "-o", os.devnull]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return r.stdout + r.stderr


if __name__ == "__main__":
    build(force=True, verbose=True)
