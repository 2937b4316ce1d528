"""Python binding of libtrees (include/trees.h): the TREES epoch step on one
B300.

The functions below carry the C names and only marshal arguments; every step
of the run executes in the CUDA library.  Device buffers are torch tensors
(``tensor.data_ptr()``), streams are ``torch.cuda.Stream`` objects or raw
handles.  The library is loaded on first use; if ``libtrees.so`` is missing
this raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtrees.so")

# status codes
TREES_OK = 0
TREES_ERR_CAPACITY = 1
TREES_ERR_EPOCH_LIMIT = 2
TREES_ERR_TIMEOUT = 3
TREES_ERR_INVALID_ARG = 4
TREES_ERR_CUDA = 5
TREES_ERR_ADMISSION = 6
TREES_ERR_STACK = 7
TREES_ERR_BUSY = 8
STATUS_NAMES = {0: "OK", 1: "CAPACITY", 2: "EPOCH_LIMIT", 3: "TIMEOUT", 4: "INVALID_ARG", 5: "CUDA",
                6: "ADMISSION", 7: "STACK", 8: "BUSY"}

# programs
TREES_PROG_FIB = 1
TREES_PROG_MERGESORT = 2
TREES_PROG_NQUEENS = 3
TREES_PROG_BFS = 4
TREES_PROG_POSTORDER = 5
TREES_PROG_PREORDER = 6
TREES_PROG_SSSP = 7
TREES_PROG_FFT = 8
TREES_PROG_USER = 9
TREES_USER_PARAMS = 4
TREES_NUM_TASK_TYPES = 13  # task types 1..13; a user program's types share this range

# schedulers
TREES_SCHED_PERSISTENT = 0
TREES_SCHED_GRAPH = 1
TREES_SCHED_HOSTLOOP = 2


class TreesError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} returned {code} ({STATUS_NAMES.get(code, '?')})")
        self.code = code


class trees_config_t(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("scheduler", ctypes.c_int32),
                ("trace", ctypes.c_int32), ("max_epochs", ctypes.c_uint32), ("trace_cap", ctypes.c_uint32),
                ("timeout_ns", ctypes.c_uint64), ("map_capacity", ctypes.c_uint64),
                ("inject_stall_epoch", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
                ("tasks_per_thread", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class trees_job_t(ctypes.Structure):
    _fields_ = [("program", ctypes.c_int32), ("n", ctypes.c_uint32), ("cutoff", ctypes.c_uint32),
                ("leaf", ctypes.c_uint32), ("keys", ctypes.c_void_p), ("scratch", ctypes.c_void_p),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("level", ctypes.c_void_p),
                ("nv", ctypes.c_int32), ("left", ctypes.c_void_p), ("right", ctypes.c_void_p),
                ("visit_epoch", ctypes.c_void_p), ("weight", ctypes.c_void_p), ("dist", ctypes.c_void_p),
                ("sched", ctypes.c_void_p), ("fft_in", ctypes.c_void_p), ("fft_out", ctypes.c_void_p),
                ("user_program", ctypes.c_void_p), ("user_type", ctypes.c_uint32), ("user_a0", ctypes.c_uint32),
                ("user_a1", ctypes.c_uint32), ("user_pad", ctypes.c_uint32),
                ("user_ptr", ctypes.c_void_p * 4), ("user_val", ctypes.c_uint64 * 4)]


class trees_stats_t(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_uint64), ("tasks", ctypes.c_uint64), ("forks", ctypes.c_uint64),
                ("joins", ctypes.c_uint64), ("maps", ctypes.c_uint64), ("peak_slots", ctypes.c_uint64),
                ("final_slots", ctypes.c_uint64), ("ns", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("error_epoch", ctypes.c_int32), ("grid_blocks", ctypes.c_int32), ("block_size", ctypes.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class trees_epoch_t(ctypes.Structure):
    _fields_ = [("cen", ctypes.c_uint32), ("lo", ctypes.c_uint32), ("hi", ctypes.c_uint32),
                ("valid", ctypes.c_uint32), ("forks", ctypes.c_uint32), ("joined", ctypes.c_uint32),
                ("maps", ctypes.c_uint32), ("ns_phase2", ctypes.c_uint32), ("t_ns", ctypes.c_uint64),
                ("ns_partition", ctypes.c_uint32), ("ns_map", ctypes.c_uint32)]


class trees_job_result_t(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("result", ctypes.c_uint64), ("tasks", ctypes.c_uint64),
                ("joins", ctypes.c_uint64), ("maps", ctypes.c_uint64), ("ns", ctypes.c_uint64),
                ("epochs", ctypes.c_uint32), ("peak_slots", ctypes.c_uint32), ("status", ctypes.c_int32),
                ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_ if f != "pad"}


class trees_tune_entry_t(ctypes.Structure):
    _fields_ = [("cfg", trees_config_t), ("ms", ctypes.c_double), ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]


_lib = None
_vp = ctypes.c_void_p
_ctxp = ctypes.c_void_p

# (name, restype, argtypes) of every exported function
_SIGNATURES = [
    ("trees_default_config", None, [ctypes.POINTER(trees_config_t)]),
    ("trees_bytes_for", ctypes.c_size_t, [ctypes.c_size_t, ctypes.POINTER(trees_config_t)]),
    ("trees_create", ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(trees_config_t), ctypes.POINTER(_ctxp)]),
    ("trees_create_on", ctypes.c_int, [_vp, ctypes.c_size_t, ctypes.POINTER(trees_config_t),
                                       ctypes.POINTER(_ctxp)]),
    ("trees_destroy", None, [_ctxp]),
    ("trees_capacity", ctypes.c_size_t, [_ctxp]),
    ("trees_geometry", ctypes.c_int, [_ctxp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
    ("trees_run", ctypes.c_int, [_ctxp, ctypes.POINTER(trees_job_t), _vp]),
    ("trees_sync", ctypes.c_int, [_ctxp]),
    ("trees_result", ctypes.c_int, [_ctxp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)]),
    ("trees_stats", ctypes.c_int, [_ctxp, ctypes.POINTER(trees_stats_t)]),
    ("trees_trace", ctypes.c_int, [_ctxp, ctypes.POINTER(trees_epoch_t), ctypes.c_size_t,
                                   ctypes.POINTER(ctypes.c_size_t)]),
    ("trees_fib", ctypes.c_int, [_ctxp, ctypes.c_uint32, ctypes.c_uint32, _vp]),
    ("trees_nqueens", ctypes.c_int, [_ctxp, ctypes.c_uint32, _vp]),
    ("trees_mergesort_u32", ctypes.c_int, [_ctxp, _vp, _vp, ctypes.c_uint32, _vp]),
    ("trees_bfs", ctypes.c_int, [_ctxp, _vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp]),
    ("trees_sssp", ctypes.c_int, [_ctxp, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp]),
    ("trees_fft", ctypes.c_int, [_ctxp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _vp]),
    ("trees_barrier_floor", ctypes.c_int, [_ctxp, ctypes.c_uint32, _vp, ctypes.POINTER(ctypes.c_double)]),
    ("trees_fib_noalloc", ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, _vp, _vp, _vp]),
    ("trees_autotune", ctypes.c_int, [ctypes.POINTER(trees_job_t), ctypes.c_size_t, ctypes.POINTER(trees_config_t),
                                      ctypes.c_int32, ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(trees_config_t),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(trees_tune_entry_t),
                                      ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    ("trees_job_slots", ctypes.c_uint64, [ctypes.POINTER(trees_job_t), ctypes.POINTER(ctypes.c_int32)]),
    ("trees_batch_run", ctypes.c_int, [_ctxp, ctypes.POINTER(trees_job_t), ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.c_int32, _vp]),
    ("trees_batch_results", ctypes.c_int, [_ctxp, ctypes.POINTER(trees_job_result_t), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_uint32)]),
    ("trees_server_create", ctypes.c_int, [ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(trees_config_t), ctypes.POINTER(_vp)]),
    ("trees_server_destroy", None, [_vp]),
    ("trees_server_submit", ctypes.c_int, [_vp, ctypes.POINTER(trees_job_t), ctypes.c_uint64,
                                           ctypes.POINTER(ctypes.c_uint64)]),
    ("trees_server_step", ctypes.c_int, [_vp, _vp]),
    ("trees_server_poll", ctypes.c_int, [_vp, ctypes.POINTER(trees_job_result_t), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32)]),
    ("trees_server_stats", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_uint64)]),
    ("trees_server_replay", ctypes.c_int, [_vp, ctypes.POINTER(trees_job_t), ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(trees_job_result_t),
                                           _vp]),
]


def lib():
    """The loaded libtrees.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1608_00571_b300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(fn, rc):
    if rc != TREES_OK:
        raise TreesError(fn, rc)
    return rc


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return int(t.data_ptr())


# ------------------------------------------------------------ C names

def trees_default_config(**overrides) -> trees_config_t:
    cfg = trees_config_t()
    lib().trees_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def trees_bytes_for(capacity_slots: int, cfg: trees_config_t | None = None) -> int:
    return int(lib().trees_bytes_for(capacity_slots, ctypes.byref(cfg) if cfg else None))


def trees_create(capacity_slots: int, cfg: trees_config_t | None = None):
    h = _ctxp()
    _check("trees_create", lib().trees_create(capacity_slots, ctypes.byref(cfg) if cfg else None, ctypes.byref(h)))
    return h


def trees_create_on(dev_buf, nbytes: int, cfg: trees_config_t | None = None):
    h = _ctxp()
    _check("trees_create_on", lib().trees_create_on(_ptr(dev_buf), nbytes, ctypes.byref(cfg) if cfg else None,
                                                    ctypes.byref(h)))
    return h


def trees_destroy(ctx) -> None:
    lib().trees_destroy(ctx)


def trees_capacity(ctx) -> int:
    return int(lib().trees_capacity(ctx))


def trees_geometry(ctx):
    g, b, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check("trees_geometry", lib().trees_geometry(ctx, ctypes.byref(g), ctypes.byref(b), ctypes.byref(s)))
    return int(g.value), int(b.value), int(s.value)


def make_job(program: int, n: int = 0, cutoff: int = 0, leaf: int = 0, keys=None, scratch=None, row_ptr=None,
             col=None, level=None, nv: int = 0, left=None, right=None, visit_epoch=None, weight=None, dist=None,
             sched=None, fft_in=None, fft_out=None, user_program=None, user_type: int = 0, user_a0: int = 0,
             user_a1: int = 0, user_ptr=(), user_val=()) -> trees_job_t:
    j = trees_job_t()
    j.program = program
    j.n = n
    j.cutoff = cutoff
    j.leaf = leaf
    j.keys = _ptr(keys)
    j.scratch = _ptr(scratch)
    j.row_ptr = _ptr(row_ptr)
    j.col = _ptr(col)
    j.level = _ptr(level)
    j.nv = nv
    j.left = _ptr(left)
    j.right = _ptr(right)
    j.visit_epoch = _ptr(visit_epoch)
    j.weight = _ptr(weight)
    j.dist = _ptr(dist)
    j.sched = _ptr(sched)
    j.fft_in = _ptr(fft_in)
    j.fft_out = _ptr(fft_out)
    if user_program is not None:  # a function of a user program library, or its address
        j.user_program = user_program if isinstance(user_program, int) else ctypes.cast(user_program,
                                                                                          ctypes.c_void_p).value
    j.user_type = user_type
    j.user_a0 = user_a0
    j.user_a1 = user_a1
    for i, v in enumerate(user_ptr):
        j.user_ptr[i] = _ptr(v)
    for i, v in enumerate(user_val):
        j.user_val[i] = v
    return j


def trees_run(ctx, job: trees_job_t, stream=None) -> int:
    return _check("trees_run", lib().trees_run(ctx, ctypes.byref(job), _stream(stream)))


def trees_sync(ctx) -> int:
    """Waits for the last run; returns its status code (does not raise)."""
    return int(lib().trees_sync(ctx))


def trees_result(ctx, slot: int = 0) -> int:
    v = ctypes.c_uint64()
    _check("trees_result", lib().trees_result(ctx, slot, ctypes.byref(v)))
    return int(v.value)


def trees_stats(ctx) -> dict:
    st = trees_stats_t()
    _check("trees_stats", lib().trees_stats(ctx, ctypes.byref(st)))
    return st.as_dict()


def trees_trace(ctx, cap: int = 1 << 16):
    buf = (trees_epoch_t * cap)()
    n = ctypes.c_size_t()
    _check("trees_trace", lib().trees_trace(ctx, buf, cap, ctypes.byref(n)))
    return [{f: int(getattr(buf[i], f)) for f, _ in trees_epoch_t._fields_ if f != "pad"} for i in range(n.value)]


def trees_fib(ctx, n: int, cutoff: int = 0, stream=None) -> int:
    return _check("trees_fib", lib().trees_fib(ctx, n, cutoff, _stream(stream)))


def trees_nqueens(ctx, n: int, stream=None) -> int:
    return _check("trees_nqueens", lib().trees_nqueens(ctx, n, _stream(stream)))


def trees_mergesort_u32(ctx, keys, scratch, n: int, stream=None) -> int:
    return _check("trees_mergesort_u32", lib().trees_mergesort_u32(ctx, _ptr(keys), _ptr(scratch), n,
                                                                   _stream(stream)))


def trees_bfs(ctx, row_ptr, col, nv: int, src: int, level, stream=None) -> int:
    return _check("trees_bfs", lib().trees_bfs(ctx, _ptr(row_ptr), _ptr(col), nv, src, _ptr(level),
                                               _stream(stream)))


def trees_sssp(ctx, row_ptr, col, weight, nv: int, src: int, dist, sched, stream=None) -> int:
    return _check("trees_sssp", lib().trees_sssp(ctx, _ptr(row_ptr), _ptr(col), _ptr(weight), nv, src, _ptr(dist),
                                                 _ptr(sched), _stream(stream)))


def trees_fft(ctx, x, out, n: int, leaf: int = 0, cutoff: int = 0, stream=None) -> int:
    return _check("trees_fft", lib().trees_fft(ctx, _ptr(x), _ptr(out), n, leaf, cutoff, _stream(stream)))


def trees_barrier_floor(ctx, iters: int = 1000, stream=None) -> float:
    us = ctypes.c_double()
    _check("trees_barrier_floor", lib().trees_barrier_floor(ctx, iters, _stream(stream), ctypes.byref(us)))
    return float(us.value)


def trees_fib_noalloc(n: int, cutoff: int, dev_result, dev_status, stream=None) -> int:
    """fib(n) without any device allocation (static 26 MiB task vector inside
    the library, at most 2^20 slots); results land in the caller's device
    buffers ``dev_result`` (uint64) and ``dev_status`` (int32).  Returns the
    host-side status; raises only through the caller's own checks."""
    return int(lib().trees_fib_noalloc(n, cutoff, _ptr(dev_result), _ptr(dev_status), _stream(stream)))


def trees_autotune(job: trees_job_t, capacity_slots: int, base: trees_config_t | None = None, reps: int = 3,
                   cache_path: str | None = None, key: str | None = None):
    """``(best config, best ms, [candidate dicts])``."""
    best = trees_config_t()
    ms = ctypes.c_double()
    cap = 32
    table = (trees_tune_entry_t * cap)()
    n = ctypes.c_int32()
    _check("trees_autotune", lib().trees_autotune(
        ctypes.byref(job), capacity_slots, ctypes.byref(base) if base else None, reps,
        cache_path.encode() if cache_path else None, key.encode() if key else None, ctypes.byref(best),
        ctypes.byref(ms), table, cap, ctypes.byref(n)))
    cands = [{"block_size": table[i].cfg.block_size, "tasks_per_thread": table[i].cfg.tasks_per_thread,
              "scheduler": table[i].cfg.scheduler, "ms": table[i].ms, "status": table[i].status}
             for i in range(n.value)]
    return best, float(ms.value), cands


def trees_job_slots(job: trees_job_t):
    """``(slots, exact)``: peak task-vector need of a job."""
    ex = ctypes.c_int32()
    v = lib().trees_job_slots(ctypes.byref(job), ctypes.byref(ex))
    return int(v), bool(ex.value)


def _job_array(jobs):
    arr = (trees_job_t * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = j
    return arr


def _u64_array(vals):
    if vals is None:
        return None
    arr = (ctypes.c_uint64 * len(vals))()
    for i, v in enumerate(vals):
        arr[i] = int(v)
    return arr


def trees_batch_run(ctx, jobs, seg_slots=None, stream=None) -> int:
    arr = _job_array(jobs)
    segs = _u64_array(seg_slots)
    return _check("trees_batch_run", lib().trees_batch_run(ctx, arr, segs, len(jobs), _stream(stream)))


def trees_batch_results(ctx, njobs: int):
    """``(status, [per-job dict], steps)``."""
    out = (trees_job_result_t * njobs)()
    steps = ctypes.c_uint32()
    rc = lib().trees_batch_results(ctx, out, njobs, ctypes.byref(steps))
    if rc in (TREES_ERR_INVALID_ARG, TREES_ERR_CUDA):
        raise TreesError("trees_batch_results", rc)
    return rc, [out[i].as_dict() for i in range(njobs)], int(steps.value)


def trees_server_create(pool_slots: int, max_jobs: int, steps_per_launch: int, cfg: trees_config_t | None = None):
    h = _vp()
    _check("trees_server_create", lib().trees_server_create(pool_slots, max_jobs, steps_per_launch,
                                                            ctypes.byref(cfg) if cfg else None, ctypes.byref(h)))
    return h


def trees_server_destroy(srv) -> None:
    lib().trees_server_destroy(srv)


def trees_server_submit(srv, job: trees_job_t, seg_slots: int = 0) -> int:
    i = ctypes.c_uint64()
    _check("trees_server_submit", lib().trees_server_submit(srv, ctypes.byref(job), seg_slots, ctypes.byref(i)))
    return int(i.value)


def trees_server_step(srv, stream=None) -> int:
    return _check("trees_server_step", lib().trees_server_step(srv, _stream(stream)))


def trees_server_poll(srv, cap: int = 4096):
    out = (trees_job_result_t * cap)()
    n = ctypes.c_int32()
    _check("trees_server_poll", lib().trees_server_poll(srv, out, cap, ctypes.byref(n)))
    return [out[i].as_dict() for i in range(n.value)]


def trees_server_stats(srv):
    q, r, L = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_uint64()
    _check("trees_server_stats", lib().trees_server_stats(srv, ctypes.byref(q), ctypes.byref(r), ctypes.byref(L)))
    return int(q.value), int(r.value), int(L.value)


def trees_server_replay(srv, jobs, arrival_s, seg_slots=None, plain: bool = False, stream=None):
    """``(latency seconds list, [per-job dict])`` of a real-time replay."""
    n = len(jobs)
    arr = _job_array(jobs)
    arrivals = (ctypes.c_double * n)(*[float(a) for a in arrival_s])
    lat = (ctypes.c_double * n)()
    res = (trees_job_result_t * n)()
    _check("trees_server_replay", lib().trees_server_replay(srv, arr, _u64_array(seg_slots), arrivals, n,
                                                            1 if plain else 0, lat, res, _stream(stream)))
    return [float(lat[i]) for i in range(n)], [res[i].as_dict() for i in range(n)]


def exported_symbols():
    """Names of the functions the binding declares (all must exist in the .so)."""
    return [name for name, _, _ in _SIGNATURES]
