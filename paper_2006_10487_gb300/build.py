"""Builds libhlbm.so in-tree for sm_103a (nvcc + g++, no cmake).

Usage: python -m paper_2006_10487_gb300.build [--force] [--debug]

--debug builds libhlbm_debug.so instead: the same sources with every kernel's
index bounds checked (HLBM_DEBUG); the binding loads it when the environment
sets HLBM_DEBUG=1.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhlbm.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libhlbm_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")

SOURCES = ["kernels.cu", "api.cu", "setup.cpp", "static_forces.cu", "adjoint.cu"]
HEADERS = ["hlbm_internal.h", "hlbm_device.h", os.path.join("..", "..", "include", "hlbm.h")]


def _cmd(src, obj, debug=False):
    defs = ["-DHLBM_DEBUG"] if debug else []
    if src.endswith(".cu"):
        return [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-pthread", *defs,
                "-c", os.path.join(CSRC, src), "-o", obj]
    return ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-pthread", "-Wall", *defs,
            f"-I{CUDA_HOME}/include", "-c", os.path.join(CSRC, src), "-o", obj]


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, debug=False):
    """Compile every translation unit (in parallel) and link libhlbm.so
    (libhlbm_debug.so, with the kernels' bounds checks, if debug)."""
    build_dir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS]
    jobs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(build_dir, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [os.path.join(CSRC, src), *headers, __file__]):
            jobs.append(_cmd(src, obj, debug))
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for res in ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs):
            if verbose or res.returncode:
                sys.stderr.write(res.stdout + res.stderr)
            if res.returncode:
                raise RuntimeError("compilation failed: " + " ".join(res.args))
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        link = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        res = subprocess.run(link, capture_output=True, text=True)
        if res.returncode:
            sys.stderr.write(res.stdout + res.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
