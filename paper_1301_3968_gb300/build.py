"""Builds libdd.so (the C-ABI library) in-tree with nvcc for sm_103a, and its debug
twin libdd_debug.so (the kernels compiled with -DDD_DEBUG: bounds checks that record
DD_ERR_ARG in the plan's device status word instead of faulting).

Translation units are compiled in parallel and linked against the static CUDA
runtime, so the library has no link-time dependency on libcuda; it loads on a
machine without a GPU and fails with DD_ERR_CUDA at its first device call.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libdd.so")
LIB_DEBUG = os.path.join(OUT_DIR, "libdd_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["dd_plan.cpp", "dd_dedisp.cu", "dd_boxcar.cu", "dd_adjoint.cu", "dd_noalloc.cu", "dd_batch.cpp",
           "dd_peak.cu", "dd_select.cpp", "dd_fused.cu"]
DEBUG_SOURCES = ["dd_dedisp.cu", "dd_fused.cu", "dd_boxcar.cu"]   # the kernels with bounds checks


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "dd.h"))
    files.append(os.path.abspath(__file__))
    return files


def _compile(src: str, verbose: bool, debug: bool = False) -> str:
    obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ("_debug" if debug else "") + ".o")
    cmd = [_nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17",
           "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if debug:
        cmd += ["-DDD_DEBUG"]
    if src.endswith(".cu"):
        cmd += ARCH + ["-lineinfo"]
        if verbose:
            cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr:
        print(res.stderr)
    return obj


def _link(objs: list[str], lib: str) -> None:
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [_nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-ldl"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.exists(LIB_DEBUG):
        t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_DEBUG))
        if all(os.path.getmtime(f) <= t for f in _deps()):
            return LIB
    jobs = [(s, False) for s in SOURCES] + [(s, True) for s in DEBUG_SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(lambda j: _compile(j[0], verbose, j[1]), jobs))
    normal = objs[:len(SOURCES)]
    dbg = dict(zip(DEBUG_SOURCES, objs[len(SOURCES):]))
    _link(normal, LIB)
    _link([dbg.get(s, o) for s, o in zip(SOURCES, normal)], LIB_DEBUG)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
