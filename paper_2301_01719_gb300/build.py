"""Builds libradtex.so in-tree with nvcc for sm_103a (GB300).

The translation units compile in parallel, then link into one shared library
next to this file.  Rebuilds only when a source or header is newer than the
library.  The checked build, libradtex_checked.so, is the same sources compiled
with RADTEX_CHECKED (every computed texel address bounds-checked on the device,
failures reported through the status word).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libradtex.so")
LIB_CHECKED = os.path.join(HERE, "libradtex_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libradtex")
    return p


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def library(checked: bool = False) -> str:
    return LIB_CHECKED if checked else LIB


def up_to_date(checked: bool = False) -> bool:
    lib = library(checked)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _flags(checked: bool, ptxas_info: bool) -> list[str]:
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                    "--expt-relaxed-constexpr"]
    if checked:
        flags += ["-DRADTEX_CHECKED"]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]
    return flags


def _compile_one(job):
    src, checked, ptxas_info = job
    obj = os.path.join(BUILD, "checked" if checked else "", os.path.basename(src) + ".o")
    cmd = [nvcc()] + _flags(checked, ptxas_info) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _link(objs, lib):
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build_variants(variants, force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> list[str]:
    """Builds the named variants (False: libradtex.so, True: the checked build),
    all their translation units compiled in one pool."""
    todo = [c for c in variants if force or not up_to_date(c)]
    if todo:
        os.makedirs(os.path.join(BUILD, "checked"), exist_ok=True)
        srcs = _sources()
        jobs = [(src, c, ptxas_info) for c in todo for src in srcs]
        with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
            results = list(ex.map(_compile_one, jobs))
        if verbose or ptxas_info:
            for obj, err in results:
                if err.strip():
                    print(f"== {os.path.relpath(obj, BUILD)}\n{err}")
        for k, c in enumerate(todo):
            _link([o for o, _ in results[k * len(srcs):(k + 1) * len(srcs)]], library(c))
    return [library(c) for c in variants]


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, checked: bool = False) -> str:
    return build_variants([checked], force, verbose, ptxas_info)[0]


def build_all(force: bool = False, verbose: bool = False) -> list[str]:
    """libradtex.so and libradtex_checked.so."""
    return build_variants([False, True], force, verbose)


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                checked="--checked" in sys.argv))
