"""In-tree build of the CUDA library ``_build/libsic.so`` for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into one shared library with the CUDA runtime linked statically, so
the library only needs the driver at run time.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsic.so")
SOURCES = ["sic_kernels.cu", "sic_api.cu", "sic_server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return [f for f in files if f.endswith((".cu", ".h", ".cuh"))]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def compile_command(src: str) -> list:
    """The nvcc command line that compiles one translation unit."""
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    return [_nvcc(), *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]


def link_command(out: str) -> list:
    """The nvcc command line that links the objects into the library."""
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    return [_nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", out, *objs]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link ``libsic.so`` if any source is newer; return its path."""
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    for src in SOURCES:
        cmd = compile_command(src)
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(" ".join(cmd) + "\n" + out.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(link_command(tmp))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
