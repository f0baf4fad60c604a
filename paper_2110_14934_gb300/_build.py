"""Build libgmm.so (sm_103a) in-tree with nvcc: the translation units compile
in parallel, then link into one shared library with the static CUDA runtime."""
from __future__ import annotations

import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libgmm.so")
UNITS = ["gmm_kernels.cu", "gmm_pool_kernel.cu", "gmm_staged.cu", "gmm_capi.cu", "gmm_pool.cu",
         "gmm_noalloc.cu", "gmm_server.cu"]
ARCH = "103a"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "gmm.h"))
    return [f for f in files if f.endswith((".cu", ".cuh", ".h"))]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def nvcc_flags(arch: str = ARCH):
    return ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo",
            f"-gencode=arch=compute_{arch},code=sm_{arch}", "-I", INCLUDE, "-I", CSRC]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link; returns the library path. Raises on failure."""
    if not force and not stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    procs = []
    objs = []
    for u in UNITS:
        obj = os.path.join(OUT, u.replace(".cu", f".{os.getpid()}.o"))
        objs.append(obj)
        cmd = ["nvcc", "-c"] + nvcc_flags() + (["-Xptxas", "-v"] if verbose else []) + \
              ["-o", obj, os.path.join(CSRC, u)]
        procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for u, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            errors.append(f"--- {u}\n{text}")
        elif verbose and text:
            print(text)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run(["nvcc", "-shared", f"-gencode=arch=compute_{ARCH},code=sm_{ARCH}", "-o", tmp]
                   + objs + ["-ldl"], check=True)
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB
