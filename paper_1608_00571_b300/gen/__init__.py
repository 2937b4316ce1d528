"""Seeded synthetic inputs for the TREES workloads (keys, R-MAT graphs, job
mixes, Poisson arrivals, binary trees).

This module is shared by the CUDA path's tests and benchmarks and by the CPU
oracle's tests; it contains no arithmetic of the task-parallel method itself.
The C source (``gen.c``) is compiled on first use with gcc into
``libtrees_gen.so`` next to it.
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_SO = os.path.join(_HERE, "libtrees_gen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libtrees_gen.so if it is missing or stale."""
    lock = os.path.join(_HERE, ".build.lock")
    with open(lock, "w") as lf:
        fcntl.flock(lf, fcntl.LOCK_EX)
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + ".tmp"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", _SRC,
                                   "-o", tmp, "-lm"])
            os.replace(tmp, _SO)
    return _SO


class _Graph(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("m", ctypes.c_int64), ("generated", ctypes.c_int64),
                ("self_loops", ctypes.c_int64), ("row_ptr", ctypes.POINTER(ctypes.c_int32)),
                ("col", ctypes.POINTER(ctypes.c_int32))]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.trees_gen_splitmix64.restype = ctypes.c_uint64
        lib.trees_gen_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.trees_gen_keys_u32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
        lib.trees_gen_rmat.restype = ctypes.c_int
        lib.trees_gen_rmat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, ctypes.POINTER(_Graph)]
        lib.trees_gen_graph_free.argtypes = [ctypes.POINTER(_Graph)]
        lib.trees_gen_weights.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_uint32, ctypes.c_void_p]
        lib.trees_gen_jobs.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
        lib.trees_gen_poisson_arrivals.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double,
                                                   ctypes.c_void_p]
        lib.trees_gen_binary_tree.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.c_void_p]
        lib.trees_gen_signal.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
        _lib = lib
    return _lib


def splitmix64(seed: int, i: int) -> int:
    """Output i (0-based) of the splitmix64 stream seeded with ``seed``."""
    return int(_load().trees_gen_splitmix64(seed, i))


def keys_u32(seed: int, n: int) -> np.ndarray:
    """``n`` uint32 keys, key i = high 32 bits of splitmix64(seed, i)."""
    out = np.empty(n, dtype=np.uint32)
    if n:
        _load().trees_gen_keys_u32(seed, n, out.ctypes.data)
    return out


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 2):
    """Undirected, deduplicated R-MAT graph as int32 CSR ``(row_ptr, col, info)``."""
    lib = _load()
    g = _Graph()
    rc = lib.trees_gen_rmat(scale, edge_factor, a, b, c, seed, ctypes.byref(g))
    if rc != 0:
        raise RuntimeError(f"trees_gen_rmat failed ({rc})")
    try:
        row_ptr = np.ctypeslib.as_array(g.row_ptr, shape=(g.nv + 1,)).copy()
        col = np.ctypeslib.as_array(g.col, shape=(max(g.m, 1),))[: g.m].copy()
    finally:
        lib.trees_gen_graph_free(ctypes.byref(g))
    info = {"scale": scale, "edge_factor": edge_factor, "a": a, "b": b, "c": c, "seed": seed,
            "nv": int(row_ptr.shape[0] - 1), "m": int(col.shape[0]), "generated": int(g.generated),
            "self_loops": int(g.self_loops)}
    return row_ptr, col, info


JOB_FIB, JOB_SORT, JOB_NQUEENS = 0, 1, 2


def jobs(seed: int, njobs: int):
    """Job mix ``(kind, param, key_seed)``; kind 0 fib(n), 1 mergesort(size), 2 N-Queens(n)."""
    kind = np.empty(njobs, dtype=np.int32)
    param = np.empty(njobs, dtype=np.int64)
    key_seed = np.empty(njobs, dtype=np.uint64)
    if njobs:
        _load().trees_gen_jobs(seed, njobs, kind.ctypes.data, param.ctypes.data, key_seed.ctypes.data)
    return kind, param, key_seed


def poisson_arrivals(seed: int, n: int, rate: float) -> np.ndarray:
    """``n`` arrival times (seconds) of a Poisson process with ``rate`` per second."""
    out = np.empty(n, dtype=np.float64)
    if n:
        _load().trees_gen_poisson_arrivals(seed, n, rate, out.ctypes.data)
    return out


def binary_tree(seed: int, nnodes: int):
    """Random binary tree ``(left, right)`` with node 0 as root, -1 = nil."""
    left = np.empty(nnodes, dtype=np.int32)
    right = np.empty(nnodes, dtype=np.int32)
    if nnodes:
        _load().trees_gen_binary_tree(seed, nnodes, left.ctypes.data, right.ctypes.data)
    return left, right


def weights(seed: int, row_ptr: np.ndarray, col: np.ndarray, wmax: int = 255) -> np.ndarray:
    """uint32 edge weights in [1, wmax] aligned with col, symmetric in (v, u)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    out = np.empty(col.shape[0], dtype=np.uint32)
    if col.size:
        _load().trees_gen_weights(seed, row_ptr.shape[0] - 1, row_ptr.ctypes.data, col.ctypes.data, wmax,
                                  out.ctypes.data)
    return out


def signal(seed: int, n: int) -> np.ndarray:
    """``n`` complex64 points, real and imaginary parts uniform on [-1, 1)."""
    out = np.empty(n, dtype=np.complex64)
    if n:
        _load().trees_gen_signal(seed, n, out.ctypes.data)
    return out
