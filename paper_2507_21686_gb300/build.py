"""Build libsph2d.so (the C-ABI library) for sm_103a with nvcc, in-tree.

Each translation unit is compiled in parallel to an object file, then linked into
``paper_2507_21686_gb300/_build/libsph2d.so``.  Rebuilds only when a source changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsph2d.so")
OPCOUNT_LIB = os.path.join(BUILD, "libsph2d_opcount.so")
SOURCES = ["sph2d_api.cu", "cells.cu", "integrals.cu", "integrals_fp64.cu", "integrals_fp32.cu",
           "backward.cu", "noalloc.cu", "surrogate.cu", "fields.cu", "hybrid.cu", "fields_p.cu", "pressure.cu", "peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsph2d")
    return cand


def source_digest() -> str:
    """SHA-256 over the library's sources, headers and flags (the build stamp)."""
    return _digest()


def _digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode() + fh.read())
    # flags with the checkout's own path left out, so that a copy elsewhere has the same digest
    h.update(" ".join(f.replace(ROOT, "<root>") for f in ARCH + FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "libsph2d.sha256")
    dig = _digest()
    if (not force and os.path.exists(LIB) and os.path.exists(OPCOUNT_LIB) and os.path.exists(stamp)
            and open(stamp).read() == dig):
        return LIB
    cc = nvcc()
    flags = FLAGS + (extra_flags or [])

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    build_opcount()
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


def build_opcount() -> str:
    """Host-only op counter of the pair formula (used for the roofline's algorithmic FLOPs)."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        raise RuntimeError("a host C++ compiler is required for the op counter")
    tmp = OPCOUNT_LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cxx, "-O1", "-std=c++17", "-shared", "-fPIC", os.path.join(CSRC, "op_count.cpp"),
                        "-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"op counter build failed:\n{r.stderr}")
    os.replace(tmp, OPCOUNT_LIB)
    return OPCOUNT_LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
