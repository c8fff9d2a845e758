"""Builds libfhmg.so in-tree (paper_1706_07632_gb300/_lib/) for sm_103a.

Host code (hbuild.cpp) is compiled with g++ and the CUDA translation units with nvcc
(-gencode arch=compute_103a,code=sm_103a), in parallel, then linked into one shared library.
No CMake; a rebuild is skipped when the library is newer than every source.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libfhmg.so")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _sources():
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                 + glob.glob(os.path.join(INCLUDE, "*.h")))
    return cu, cpp, hdr


def _up_to_date(deps):
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    cu, cpp, hdr = _sources()
    if not force and _up_to_date(cu + cpp + hdr + [__file__]):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    objs, procs = [], []
    for src in cu:
        obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
        cmd = [NVCC] + ARCH + NVCC_FLAGS + ["-c", src, "-o", obj]
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for src in cpp:
        obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
        cmd = ["g++"] + CXX_FLAGS + ["-c", src, "-o", obj]
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if verbose or pr.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + out.decode(errors="replace"))
        if pr.returncode:
            failed.append(cmd[-3])
    if failed:
        raise RuntimeError("compilation failed: " + ", ".join(failed))
    tmp = LIB + ".tmp"
    cmd = [NVCC] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
