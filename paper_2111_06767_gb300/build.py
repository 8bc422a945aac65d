"""Build the CUDA library libdg_elliptic.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel to `_build/`, then linked into
`paper_2111_06767_gb300/libdg_elliptic.so`. Host code is portable C++17 (x86_64 and aarch64).
Run `python paper_2111_06767_gb300/build.py` (by path: importing the package loads the library);
`--debug` builds the bounds-checked variant libdg_elliptic_debug.so (loaded with DG_DEBUG_BUILD=1).
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(os.path.dirname(PKG), "_build")
LIB = os.path.join(PKG, "libdg_elliptic.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
SOURCES = ["lgl.cpp", "dg_apply.cu", "schwarz.cu", "mg.cu", "blas.cu", "puncture.cu", "setup.cu", "solver.cu",
           "capi.cu", "serve.cpp", "noalloc.cu", "tc_gemm.cu", "autotune.cu",
           "lin_inverse.cu", "curved.cu", "krylov_dev.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


DEBUG_BUILD = os.path.join(os.path.dirname(PKG), "_build_debug")
DEBUG_LIB = os.path.join(PKG, "libdg_elliptic_debug.so")


def _flags(verbose_ptxas: bool = False, debug: bool = False):
    f = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "--expt-relaxed-constexpr", "-I" + os.path.join(os.path.dirname(PKG), "include")]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    if debug:
        f += ["-DDG_BOUNDS_CHECK"]
    return f


def _compile(src: str, verbose_ptxas: bool, debug: bool = False) -> str:
    obj = os.path.join(DEBUG_BUILD if debug else BUILD, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    lang = ["-x", "cu"] if src.endswith(".cu") else ["-x", "c++"]
    cmd = [nvcc()] + lang + _flags(verbose_ptxas, debug) + ["-c", path, "-o", obj]
    deps = [path] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(os.path.dirname(PKG), "include", "dg_elliptic.h"))
    if os.path.exists(obj) and all(os.path.getmtime(obj) >= os.path.getmtime(d) for d in deps):
        return obj
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if verbose_ptxas:
        sys.stderr.write(res.stderr)
    return obj


def build(verbose_ptxas: bool = False, jobs: int | None = None, debug: bool = False) -> str:
    """Release library (libdg_elliptic.so); with debug=True the bounds-checked variant
    (libdg_elliptic_debug.so, -DDG_BOUNDS_CHECK), built apart in _build_debug/."""
    out_dir, lib = (DEBUG_BUILD, DEBUG_LIB) if debug else (BUILD, LIB)
    os.makedirs(out_dir, exist_ok=True)
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with concurrent.futures.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas, debug), SOURCES))
    if not os.path.exists(lib) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        cmd = [nvcc(), ARCH, "-shared", "-o", lib] + objs + ["-lpthread"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    return lib


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, debug="--debug" in sys.argv))
