"""CPU oracle for the TREES epoch step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``oracle.c`` (plain sequential C: the
recursive definitions of each task program and a Task Vector Machine
simulator that follows the paper's Phase 1/2/3 epoch loop, Sec. 4.3 and 5.2)
through ctypes.  It shares no code with the CUDA path and imports nothing
from it.
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

FIB, MERGESORT, BFS, NQUEENS, POSTORDER, PREORDER, FFT = 0, 1, 2, 3, 4, 5, 6


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so if it is missing or stale."""
    with open(os.path.join(_HERE, ".build.lock"), "w") as lf:
        fcntl.flock(lf, fcntl.LOCK_EX)
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + ".tmp"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _SO)
    return _SO


class Epoch(ctypes.Structure):
    _fields_ = [("cen", ctypes.c_uint32), ("lo", ctypes.c_uint32), ("hi", ctypes.c_uint32),
                ("valid", ctypes.c_uint32), ("forks", ctypes.c_uint32), ("joined", ctypes.c_uint32),
                ("maps", ctypes.c_uint32)]


class _Params(ctypes.Structure):
    _fields_ = [("program", ctypes.c_int), ("fib_n", ctypes.c_uint32), ("fib_cutoff", ctypes.c_uint32),
                ("keys", ctypes.c_void_p), ("nkeys", ctypes.c_int64), ("leaf", ctypes.c_int64),
                ("nv", ctypes.c_int32), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("level", ctypes.c_void_p), ("src", ctypes.c_int32), ("nq_n", ctypes.c_int32),
                ("nnodes", ctypes.c_int32), ("left", ctypes.c_void_p), ("right", ctypes.c_void_p),
                ("visit_epoch", ctypes.c_void_p), ("max_epochs", ctypes.c_uint64),
                ("fft_n", ctypes.c_int64), ("fft_leaf", ctypes.c_int64), ("fft_cutoff", ctypes.c_int64),
                ("fft_x", ctypes.c_void_p), ("fft_X", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_uint64), ("tasks", ctypes.c_uint64), ("forks", ctypes.c_uint64),
                ("joins", ctypes.c_uint64), ("maps", ctypes.c_uint64), ("peak_slots", ctypes.c_uint64),
                ("root_result", ctypes.c_uint64), ("final_slots", ctypes.c_uint64),
                ("err", ctypes.c_int32)]


def _bind(lib):
    """Declares the C signatures on a loaded oracle library and returns it."""
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.oracle_fib.restype = ctypes.c_uint64
    lib.oracle_fib.argtypes = [ctypes.c_uint32, u64p]
    lib.oracle_fib_task_counts.argtypes = [ctypes.c_uint32, ctypes.c_uint32, u64p, u64p]
    lib.oracle_mergesort_u32.restype = ctypes.c_int
    lib.oracle_mergesort_u32.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]
    lib.oracle_bfs.restype = ctypes.c_int64
    lib.oracle_bfs.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                               ctypes.c_void_p]
    lib.oracle_sssp_dijkstra.restype = ctypes.c_int64
    lib.oracle_sssp_dijkstra.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_void_p]
    lib.oracle_sssp_worklist.restype = ctypes.c_int
    lib.oracle_sssp_worklist.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_void_p, u64p, u64p]
    lib.oracle_nqueens.restype = ctypes.c_uint64
    lib.oracle_nqueens.argtypes = [ctypes.c_int, u64p, u64p]
    lib.oracle_dft.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_dft_at.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    lib.oracle_tvm_run.restype = ctypes.c_int
    lib.oracle_tvm_run.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(Epoch), ctypes.c_uint64,
                                   ctypes.POINTER(_Stats)]
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_SO))
    return _lib


# ------------------------------------------------------------ plain definitions

def fib(n: int):
    """Recursive Fibonacci: ``(F(n), number of calls)``."""
    calls = ctypes.c_uint64()
    v = _load().oracle_fib(n, ctypes.byref(calls))
    return int(v), int(calls.value)


def fib_task_counts(n: int, cutoff: int = 0):
    """``(fib tasks, join tasks)`` of the fib task tree with leaves n<2 or n<=cutoff."""
    t, j = ctypes.c_uint64(), ctypes.c_uint64()
    _load().oracle_fib_task_counts(n, cutoff, ctypes.byref(t), ctypes.byref(j))
    return int(t.value), int(j.value)


def mergesort(keys: np.ndarray, leaf: int = 1024) -> np.ndarray:
    """Top-down mergesort of uint32 keys with the method's split rule; returns a sorted copy."""
    out = np.ascontiguousarray(keys, dtype=np.uint32).copy()
    rc = _load().oracle_mergesort_u32(out.ctypes.data, out.shape[0], leaf)
    if rc != 0:
        raise RuntimeError(f"oracle_mergesort_u32 failed ({rc})")
    return out


def bfs(row_ptr: np.ndarray, col: np.ndarray, src: int = 0):
    """FIFO-queue BFS: ``(level int32 array, reached count)``."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    nv = row_ptr.shape[0] - 1
    level = np.empty(nv, dtype=np.int32)
    reached = _load().oracle_bfs(nv, row_ptr.ctypes.data, col.ctypes.data if col.size else None, src,
                                 level.ctypes.data)
    return level, int(reached)


SSSP_INF = np.iinfo(np.uint64).max  # distance of an unreachable vertex


def _csr_args(row_ptr, col, weight):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    weight = np.ascontiguousarray(weight, dtype=np.uint32)
    assert weight.shape == col.shape
    return row_ptr, col, weight


def sssp_dijkstra(row_ptr: np.ndarray, col: np.ndarray, weight: np.ndarray, src: int = 0):
    """Dijkstra with a binary heap: ``(dist uint64 array, reached count)``;
    unreachable vertices hold SSSP_INF."""
    row_ptr, col, weight = _csr_args(row_ptr, col, weight)
    nv = row_ptr.shape[0] - 1
    dist = np.empty(nv, dtype=np.uint64)
    reached = _load().oracle_sssp_dijkstra(nv, row_ptr.ctypes.data, col.ctypes.data if col.size else None,
                                           weight.ctypes.data if weight.size else None, src, dist.ctypes.data)
    if reached < 0:
        raise MemoryError("oracle_sssp_dijkstra")
    return dist, int(reached)


def sssp_worklist(row_ptr: np.ndarray, col: np.ndarray, weight: np.ndarray, src: int = 0):
    """The worklist relaxation of Sec. 6.3, sequential: ``(dist, rounds, relaxed vertices)``."""
    row_ptr, col, weight = _csr_args(row_ptr, col, weight)
    nv = row_ptr.shape[0] - 1
    dist = np.empty(nv, dtype=np.uint64)
    rounds, relaxed = ctypes.c_uint64(), ctypes.c_uint64()
    rc = _load().oracle_sssp_worklist(nv, row_ptr.ctypes.data, col.ctypes.data if col.size else None,
                                      weight.ctypes.data if weight.size else None, src, dist.ctypes.data,
                                      ctypes.byref(rounds), ctypes.byref(relaxed))
    if rc != 0:
        raise MemoryError("oracle_sssp_worklist")
    return dist, int(rounds.value), int(relaxed.value)


def nqueens(n: int):
    """Backtracking N-Queens: ``(solutions, row tasks, join tasks)``."""
    r, j = ctypes.c_uint64(), ctypes.c_uint64()
    v = _load().oracle_nqueens(n, ctypes.byref(r), ctypes.byref(j))
    return int(v), int(r.value), int(j.value)


def _complex_in(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def dft(x) -> np.ndarray:
    """The discrete Fourier transform by its definition, O(n^2), fp64:
    ``X[k] = sum_j x[j] exp(-2 pi i j k / n)``."""
    x = _complex_in(x)
    X = np.empty_like(x)
    if x.size:
        _load().oracle_dft(x.shape[0], x.ctypes.data, X.ctypes.data)
    return X


def dft_at(x, ks) -> np.ndarray:
    """Outputs ``X[k]`` of the definition for the indices ``ks`` only, O(n) each."""
    x = _complex_in(x)
    ks = np.asarray(ks, dtype=np.int64).reshape(-1)
    out = np.empty(ks.shape[0], dtype=np.complex128)
    buf = np.empty(2, dtype=np.float64)
    for i, k in enumerate(ks):
        _load().oracle_dft_at(x.shape[0], x.ctypes.data, int(k), buf.ctypes.data)
        out[i] = complex(buf[0], buf[1])
    return out


# ------------------------------------------------------------ TVM simulator

def tvm_run(program: int, *, fib_n: int = 0, fib_cutoff: int = 0, keys: np.ndarray | None = None,
            leaf: int = 1024, row_ptr=None, col=None, src: int = 0, nq_n: int = 0, left=None, right=None,
            x=None, fft_leaf: int = 16, fft_cutoff: int = 0, max_epochs: int = 1 << 20,
            trace_cap: int = 1 << 16):
    """Runs one program on the sequential TVM simulator.

    Returns a dict with ``stats`` (epochs, tasks, forks, joins, maps,
    peak_slots, root_result), ``trace`` (structured array, one row per epoch:
    cen, lo, hi, valid, forks, joined, maps) and the program's output
    (``keys`` sorted in place on a copy, ``level``, ``visit_epoch``, or the
    FFT's output ``X`` as complex128).
    """
    lib = _load()
    p = _Params()
    p.program = program
    p.fib_n = fib_n
    p.fib_cutoff = fib_cutoff
    p.max_epochs = max_epochs
    p.leaf = leaf
    keep = []
    out = {}
    if program == MERGESORT:
        k = np.ascontiguousarray(keys, dtype=np.uint32).copy()
        keep.append(k)
        p.keys = k.ctypes.data if k.size else None
        p.nkeys = k.shape[0]
        out["keys"] = k
    if program == BFS:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        lv = np.empty(rp.shape[0] - 1, dtype=np.int32)
        keep += [rp, cl, lv]
        p.nv = rp.shape[0] - 1
        p.row_ptr = rp.ctypes.data
        p.col = cl.ctypes.data if cl.size else None
        p.level = lv.ctypes.data
        p.src = src
        out["level"] = lv
    if program == NQUEENS:
        p.nq_n = nq_n
    if program in (POSTORDER, PREORDER):
        lf = np.ascontiguousarray(left, dtype=np.int32)
        rt = np.ascontiguousarray(right, dtype=np.int32)
        ve = np.empty(lf.shape[0], dtype=np.int32)
        keep += [lf, rt, ve]
        p.nnodes = lf.shape[0]
        p.left = lf.ctypes.data if lf.size else None
        p.right = rt.ctypes.data if rt.size else None
        p.visit_epoch = ve.ctypes.data if ve.size else None
        out["visit_epoch"] = ve
    if program == FFT:
        xi = _complex_in(x)
        Xo = np.zeros_like(xi)
        keep += [xi, Xo]
        p.fft_n = xi.shape[0]
        p.fft_leaf = fft_leaf
        p.fft_cutoff = fft_cutoff
        p.fft_x = xi.ctypes.data
        p.fft_X = Xo.ctypes.data
        out["X"] = Xo
    trace = (Epoch * trace_cap)()
    st = _Stats()
    rc = lib.oracle_tvm_run(ctypes.byref(p), trace, trace_cap, ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"oracle_tvm_run failed ({rc})")
    n = min(int(st.epochs), trace_cap)
    dt = np.dtype([(f, np.uint32) for f, _ in Epoch._fields_])
    arr = np.frombuffer(trace, dtype=dt, count=n).copy()
    out["stats"] = {f: int(getattr(st, f)) for f, _ in _Stats._fields_ if f != "err"}
    out["trace"] = arr
    return out


# ------------------------------------------------------------ the user-program example

def chunk_sum_tree(n: int, chunk: int, arity: int):
    """The task tree of the chunked-sum example program, by its definition:
    SUM(lo, hi) over a range of at most ``chunk`` keys is a leaf (one map
    unit, or an emit of 0 when empty); a longer range has
    k = min(arity, ceil(len / chunk)) children over the parts
    [lo + len*i//k, lo + len*(i+1)//k) and a join.  Returns the counts and
    the per-epoch trace the task vector machine gives it: the fork levels
    0..D (every task of depth d in one range), then the join ranges revisited
    from depth D-1 back to 0 (Sec. 4.3)."""
    levels = []  # per depth: list of (lo, hi)

    def walk(lo, hi, d):
        while len(levels) <= d:
            levels.append([])
        levels[d].append((lo, hi))
        ln = hi - lo
        if ln > chunk:
            k = min(arity, -(-ln // chunk))
            for i in range(k):
                walk(lo + ln * i // k, lo + ln * (i + 1) // k, d + 1)

    walk(0, n, 0)
    D = len(levels) - 1
    internal = [sum(1 for lo, hi in lv if hi - lo > chunk) for lv in levels]
    maps = [sum(1 for lo, hi in lv if 0 < hi - lo <= chunk) for lv in levels]
    starts = [0]
    for lv in levels:
        starts.append(starts[-1] + len(lv))
    trace = []
    for d in range(D + 1):  # fork levels
        forks = len(levels[d + 1]) if d < D else 0
        trace.append({"cen": d, "lo": starts[d], "hi": starts[d + 1], "valid": len(levels[d]), "forks": forks,
                      "joined": int(internal[d] > 0), "maps": maps[d]})
    for d in range(D - 1, -1, -1):  # join ranges, deepest first
        trace.append({"cen": d, "lo": starts[d], "hi": starts[d + 1], "valid": internal[d], "forks": 0,
                      "joined": 0, "maps": 0})
    stats = {"epochs": len(trace), "tasks": sum(t["valid"] for t in trace), "joins": sum(internal),
             "maps": sum(maps), "forks": sum(len(lv) for lv in levels[1:]), "peak_slots": starts[-1],
             "final_slots": 0}
    return stats, trace
