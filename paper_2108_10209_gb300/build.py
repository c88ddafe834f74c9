"""Builds the sm_103a library ``libn2f.so`` in-tree (objects under ``_build/``).

Every translation unit is compiled by nvcc for ``compute_103a``/``sm_103a`` in parallel and
linked into one shared library that exports the C ABI of ``include/n2f.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libn2f.so")
# the checked build: the same sources with N2F_CHECKED (bounds-checked kernel indexes)
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libn2f_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
SOURCES = ["kernels_basic.cu", "kernels_simt.cu", "conv_tc.cu", "wgrad_tc.cu", "tc_probe.cu",
           "trainer.cpp", "api.cpp", "noalloc.cu"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2,-pthread",
         "-I" + os.path.join(ROOT, "include")]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "n2f.h"))
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, checked: bool = False) -> str:
    obj = os.path.join(BUILD_CHECKED if checked else BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC, *ARCH, *FLAGS] + (["-DN2F_CHECKED"] if checked else [])
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    cmd += ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds libn2f.so, or with checked=True libn2f_checked.so; returns its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps():
        return lib
    os.makedirs(BUILD_CHECKED if checked else BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, checked), SOURCES))
    tmp = lib + ".tmp"
    cmd = [NVCC, *ARCH, "-shared", "-Xcompiler", "-pthread", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv)
