"""Build the in-tree CUDA library ``_lib/liblbm.so`` for GB300 (sm_103a).

Each translation unit is compiled in parallel with nvcc, then linked into one
shared library with the C ABI of ``include/lbm.h``.  Run ``python -m
paper_1608_06345_gb300.build`` or call :func:`build`.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "liblbm.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

# (source, extra defines): step_inst.cu is built once per (lattice, precision)
SOURCES = [("lbm_api.cu", []), ("lattice_table.cpp", []), ("lbm_slab.cpp", []), ("lbm_noalloc.cu", []),
           ("lbm_pool.cu", [])] + [
    ("step_inst.cu", [f"-DLBM_LAT={lat}", f"-DLBM_PREC={prec}"]) for lat in (0, 1) for prec in (0, 1, 2, 3)]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-I", CSRC, "-I", INCLUDE]


def _stamp():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lbm.h"), __file__]
    return max(os.path.getmtime(f) for f in files if os.path.isfile(f))


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    """Compile (if stale) and return the path of liblbm.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _stamp() and not extra_flags:
        return LIB
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    extra = list(extra_flags or [])

    def compile_one(item):
        src, defs = item
        tag = "".join(d.split("=")[1] for d in defs)
        obj = os.path.join(obj_dir, os.path.splitext(src)[0] + tag + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, *defs, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):  # host code: no contraction, so the double-double sums stay exact
            cmd = [NVCC, *FLAGS, *defs, *extra, "-Xcompiler", "-ffp-contract=off", "-x", "c++", "-c",
                   os.path.join(CSRC, src), "-o", obj]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{p.stdout}\n{p.stderr}")
        if verbose and (p.stdout or p.stderr):
            sys.stderr.write(p.stdout + p.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None))
