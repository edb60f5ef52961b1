"""Builds the in-tree CUDA library ``libtrtr.so`` for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared object next to
this file.  No cmake, no torch build machinery; only nvcc (which cross-compiles without a
GPU).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtrtr.so")
# debug build whose kernels check their memory accesses (TRTR_BOUNDS_CHECK=1)
LIB_CHECKED = os.path.join(HERE, "libtrtr_checked.so")

SOURCES = ["trtr_api.cu", "trtr_step.cu", "trtr_step2.cu", "trtr_aux.cu", "trtr_noalloc.cu", "trtr_batch.cu",
           "trtr_adjoint.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                     "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libtrtr.so")
    return p


def _deps() -> list[str]:
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "trtr.h"))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build_library(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
                  out: str | None = None, checked: bool = False) -> str:
    """Compile and link libtrtr.so (or `out`); returns its path.  Raises on any compiler error.
    checked=True builds the bounds-checked debug library libtrtr_checked.so instead."""
    default = LIB_CHECKED if checked else LIB
    if not force and out is None and up_to_date(default):
        return default
    objdir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(objdir, exist_ok=True)
    cc = nvcc()
    flags = NVCC_FLAGS + (["-DTRTR_BOUNDS_CHECK=1"] if checked else []) + (extra_flags or [])
    procs = []
    objs = []
    for s in SOURCES:
        obj = os.path.join(objdir, s.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc, *flags, "-c", os.path.join(CSRC, s), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for s, p in procs:
        log, _ = p.communicate()
        if verbose and log:
            sys.stderr.write(log.decode(errors="replace"))
        if p.returncode != 0:
            errors.append(f"{s}:\n{log.decode(errors='replace')}")
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    target = out or default
    tmp = target + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    # python build.py [-v] [--ptxas] [--checked] [-DNAME=VALUE ...]: a forced rebuild; -D options
    # set the kernels' compile-time geometry switches (TRTR_STEP_*, TRTR_STEP2_*)
    v = "-v" in sys.argv
    extra = (["-Xptxas", "-v"] if "--ptxas" in sys.argv else []) + [a for a in sys.argv[1:] if a.startswith("-D")]
    print(build_library(force=True, verbose=v or "--ptxas" in sys.argv, extra_flags=extra or None,
                        checked="--checked" in sys.argv))
