"""Builds libtrees.so (the CUDA library behind include/trees.h) in-tree with
nvcc for sm_103a.  Used by ``__graft_entry__.build()`` and by the binding when
the library is missing or older than its sources."""
from __future__ import annotations

import concurrent.futures
import fcntl
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libtrees.so")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC,-O2", "-shared",
]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "trees_impl", "*.cuh"))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA/C++ source under csrc/ into libtrees.so."""
    with open(os.path.join(HERE, ".build.lock"), "w") as lf:
        fcntl.flock(lf, fcntl.LOCK_EX)
        if not force and not stale():
            return LIB
        objdir = os.path.join(HERE, "_build")
        os.makedirs(objdir, exist_ok=True)
        flags = [f for f in NVCC_FLAGS if f != "-shared"]

        def compile_one(src):
            obj = os.path.join(objdir, os.path.basename(src) + ".o")
            cmd = ["nvcc", *flags, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd))
            subprocess.check_call(cmd)
            return obj

        srcs = sources()
        with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
            objs = list(ex.map(compile_one, srcs))
        tmp = LIB + ".tmp"
        link = ["nvcc", "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp, *objs, "-lcuda"]
        if verbose:
            print(" ".join(link))
        subprocess.check_call(link)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)


def build_program(source: str, output: str, force: bool = False) -> str:
    """Compiles a user task program (a .cu file written against
    include/trees_program.cuh, ending in TREES_DEFINE_PROGRAM) into the
    shared library ``output`` with the library's own flags and the public
    include directory alone on the include path, unless it is newer than its
    source and the SDK headers.  Returns ``output``."""
    deps = [source] + glob.glob(os.path.join(INCLUDE, "*")) + glob.glob(os.path.join(INCLUDE, "trees_impl", "*"))
    if not force and os.path.exists(output) and all(os.path.getmtime(output) >= os.path.getmtime(d) for d in deps):
        return output
    tmp = output + ".tmp"
    subprocess.check_call(["nvcc", *NVCC_FLAGS, "-I", INCLUDE, source, "-o", tmp])
    os.replace(tmp, output)
    return output
