"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

All workloads are integer, so every comparison is exact: results, task and
epoch counts, and the per-epoch trace (epoch number, NDRange, valid tasks,
forks, join flag) against the TVM simulator.  Slot *contents* are not
compared across blocks (the order of the per-block atomics is not fixed),
but the ranges are: they depend only on the counts.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1608_00571_b300 as T
from paper_1608_00571_b300 import gen

pytestmark = pytest.mark.gpu

SCHEDS = [T.TREES_SCHED_PERSISTENT, T.TREES_SCHED_GRAPH, T.TREES_SCHED_HOSTLOOP]
TRACE_FIELDS = ("cen", "lo", "hi", "valid", "forks", "joined")


class Ctx:
    def __init__(self, cap, **cfg):
        c = T.trees_default_config(**cfg)
        self.h = T.trees_create(cap, c)

    def __enter__(self):
        return self.h

    def __exit__(self, *a):
        T.trees_destroy(self.h)


def run(ctx, job):
    T.trees_run(ctx, job, torch.cuda.current_stream())
    return T.trees_sync(ctx)


def check_trace(ctx, sim, fields=TRACE_FIELDS):
    tr = T.trees_trace(ctx)
    st = sim["trace"]
    assert len(tr) == len(st)
    for i, (g, o) in enumerate(zip(tr, st)):
        for f in fields:
            assert g[f] == int(o[f]), (i, f, g, o)


def dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


# ------------------------------------------------------------------ fib

@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("bs", [128, 256, 512, 1024])
@pytest.mark.parametrize("tpt", [1, 2, 4])
def test_fib20(sched, bs, tpt):
    sim = oracle.tvm_run(oracle.FIB, fib_n=20)
    with Ctx(1 << 16, scheduler=sched, block_size=bs, tasks_per_thread=tpt, trace=1) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_FIB, n=20)) == T.TREES_OK
        assert T.trees_result(ctx, 0) == 6765
        st = T.trees_stats(ctx)
        for k in ("epochs", "tasks", "forks", "joins", "peak_slots", "final_slots"):
            assert st[k] == sim["stats"][k], k
        check_trace(ctx, sim)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 7, 16, 24])
def test_fib_small(n):
    sim = oracle.tvm_run(oracle.FIB, fib_n=n)
    with Ctx(1 << 20, trace=1) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_FIB, n=n)) == T.TREES_OK
        assert T.trees_result(ctx, 0) == oracle.fib(n)[0]
        st = T.trees_stats(ctx)
        assert (st["epochs"], st["tasks"]) == (sim["stats"]["epochs"], sim["stats"]["tasks"])
        check_trace(ctx, sim)


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("n,c", [(20, 12), (25, 12), (12, 12), (28, 20)])
def test_fib_cutoff(sched, n, c):
    sim = oracle.tvm_run(oracle.FIB, fib_n=n, fib_cutoff=c)
    with Ctx(1 << 20, scheduler=sched, trace=1) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_FIB, n=n, cutoff=c)) == T.TREES_OK
        assert T.trees_result(ctx, 0) == oracle.fib(n)[0]
        st = T.trees_stats(ctx)
        assert (st["epochs"], st["tasks"], st["joins"]) == \
            (sim["stats"]["epochs"], sim["stats"]["tasks"], sim["stats"]["joins"])
        check_trace(ctx, sim)


# ------------------------------------------------------------------ N-Queens

@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("n", list(range(1, 12)))
def test_nqueens(sched, n):
    sim = oracle.tvm_run(oracle.NQUEENS, nq_n=n)
    with Ctx(1 << 20, scheduler=sched, trace=1) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_NQUEENS, n=n)) == T.TREES_OK
        assert T.trees_result(ctx, 0) == oracle.nqueens(n)[0]
        st = T.trees_stats(ctx)
        for k in ("epochs", "tasks", "forks", "joins", "peak_slots", "final_slots"):
            assert st[k] == sim["stats"][k], k
        check_trace(ctx, sim)


# ------------------------------------------------------------------ mergesort

@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("n", [0, 1, 5, 1024, 1025, 3000, 4096, 4097, 12345, 100000, (1 << 20) + 3])
def test_mergesort(sched, n):
    keys = gen.keys_u32(100 + n, n)
    sim = oracle.tvm_run(oracle.MERGESORT, keys=keys)
    d = dev_u32(keys)
    scratch = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    with Ctx(1 << 16, scheduler=sched, trace=1) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_MERGESORT, n=n, keys=d, scratch=scratch)) == T.TREES_OK
        assert np.array_equal(host_u32(d), np.sort(keys))
        assert np.array_equal(host_u32(d), sim["keys"])
        st = T.trees_stats(ctx)
        for k in ("epochs", "tasks", "forks", "joins", "maps", "final_slots"):
            assert st[k] == sim["stats"][k], k
        check_trace(ctx, sim, TRACE_FIELDS + ("maps",))


@pytest.mark.parametrize("sched", [T.TREES_SCHED_PERSISTENT, T.TREES_SCHED_GRAPH])
@pytest.mark.parametrize("bs", [128, 256, 512, 1024])
@pytest.mark.parametrize("n", [5000, 100000, (1 << 20) + 3])
def test_mergesort_block_sizes(sched, bs, n):
    keys = gen.keys_u32(7 * n + bs, n)
    d = dev_u32(keys)
    with Ctx(1 << 16, scheduler=sched, block_size=bs, timeout_ns=200_000_000) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_MERGESORT, n=n, keys=d)) == T.TREES_OK
        assert np.array_equal(host_u32(d), np.sort(keys))


@pytest.mark.parametrize("sched", [T.TREES_SCHED_PERSISTENT, T.TREES_SCHED_GRAPH])
@pytest.mark.parametrize("layout", ["keys_offset", "both_offset", "sorted", "reversed", "two_values"])
@pytest.mark.parametrize("n", [300001, (1 << 19) + 2])
def test_mergesort_alignment_and_order(sched, layout, n):
    """Arrays that are only 4-byte aligned (the merge stages fall back to plain
    loads for one or both buffers) and inputs whose merge tiles read all keys
    from one run (sorted, reversed) or from long runs of equal keys."""
    keys = gen.keys_u32(31 + n, n)
    if layout == "sorted":
        keys = np.sort(keys)
    elif layout == "reversed":
        keys = np.sort(keys)[::-1].copy()
    elif layout == "two_values":
        keys = (keys & 1) * np.uint32(0xFFFFFFFF)
    keys = keys.astype(np.uint32)
    kb = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    sb = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    d = kb[1:] if layout in ("keys_offset", "both_offset") else kb[:n]
    sc = sb[1:] if layout == "both_offset" else sb[:n]
    d.copy_(torch.from_numpy(keys.view(np.int32)))
    with Ctx(1 << 16, scheduler=sched, timeout_ns=500_000_000) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_MERGESORT, n=n, keys=d, scratch=sc)) == T.TREES_OK
        assert np.array_equal(host_u32(d), np.sort(keys))
        if layout in ("keys_offset", "both_offset"):
            assert int(kb[0].item()) == 0  # nothing written in front of the array


@pytest.mark.parametrize("leaf", [1, 3, 64, 1000])
def test_mergesort_leaf_sizes_and_duplicates(leaf):
    rng = np.random.default_rng(leaf)
    keys = rng.integers(0, 7, size=20000).astype(np.uint32)
    keys[::97] = 0xFFFFFFFF
    sim = oracle.tvm_run(oracle.MERGESORT, keys=keys, leaf=leaf)
    d = dev_u32(keys)
    with Ctx(1 << 17, trace=1) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_MERGESORT, n=keys.size, keys=d, leaf=leaf)) == T.TREES_OK
        assert np.array_equal(host_u32(d), sim["keys"])
        check_trace(ctx, sim, TRACE_FIELDS + ("maps",))


# ------------------------------------------------------------------ BFS

def random_graph(nv, p, seed):
    rng = np.random.default_rng(seed)
    a = np.triu(rng.random((nv, nv)) < p, 1)
    a = a | a.T
    row_ptr = np.zeros(nv + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum(a.sum(1))
    col = np.concatenate([np.nonzero(a[i])[0] for i in range(nv)] + [np.zeros(0, int)]).astype(np.int32)
    return row_ptr, col


def bfs_gpu(ctx, row_ptr, col, src):
    rp = torch.from_numpy(row_ptr).cuda()
    cl = torch.from_numpy(col if col.size else np.zeros(1, np.int32)).cuda()
    lv = torch.empty(row_ptr.size - 1, dtype=torch.int32, device="cuda")
    status = run(ctx, T.make_job(T.TREES_PROG_BFS, n=src, row_ptr=rp, col=cl, level=lv, nv=row_ptr.size - 1))
    return status, lv.cpu().numpy()


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("nv,p,seed", [(1, 0.0, 0), (50, 0.0, 1), (64, 0.05, 2), (300, 0.02, 3), (2000, 0.004, 4)])
def test_bfs_random(sched, nv, p, seed):
    row_ptr, col = random_graph(nv, p, seed)
    sim = oracle.tvm_run(oracle.BFS, row_ptr=row_ptr, col=col, src=0)
    with Ctx(1 << 16, scheduler=sched, trace=1) as ctx:
        status, level = bfs_gpu(ctx, row_ptr, col, 0)
        assert status == T.TREES_OK
        assert np.array_equal(level, sim["level"])
        assert np.array_equal(level, oracle.bfs(row_ptr, col, 0)[0])
        st = T.trees_stats(ctx)
        assert (st["epochs"], st["tasks"]) == (sim["stats"]["epochs"], sim["stats"]["tasks"])
        check_trace(ctx, sim)


@pytest.mark.parametrize("scale", [10, 14, 16])
def test_bfs_rmat(scale):
    row_ptr, col, _ = gen.rmat(scale, 16, seed=2)
    sim = oracle.tvm_run(oracle.BFS, row_ptr=row_ptr, col=col, src=0)
    with Ctx(1 << (scale + 1), trace=1) as ctx:
        status, level = bfs_gpu(ctx, row_ptr, col, 0)
        assert status == T.TREES_OK
        assert np.array_equal(level, sim["level"])
        check_trace(ctx, sim)


@pytest.mark.parametrize("bs,tpt,grid", [(512, 1, 0), (512, 1, 2), (256, 2, 3), (1024, 1, 2), (128, 2, 0)])
def test_bfs_capacity_edge_and_buffer_flushes(bs, tpt, grid):
    """BFS forks one visit task per reached vertex, from the flushes of the block parts' candidate
    buffers (with two or three grid blocks every part flushes many times an epoch): a task vector
    one slot short of the peak is a capacity error and the context stays usable; the peak itself
    reproduces the oracle's levels and per-epoch trace."""
    row_ptr, col, _ = gen.rmat(16, 16, seed=5)
    sim = oracle.tvm_run(oracle.BFS, row_ptr=row_ptr, col=col, src=0)
    peak = sim["stats"]["peak_slots"]
    cfg = dict(block_size=bs, tasks_per_thread=tpt, trace=1)
    if grid:
        cfg["grid_blocks"] = grid
    small_rp, small_col, _ = gen.rmat(10, 16, seed=6)
    small = oracle.tvm_run(oracle.BFS, row_ptr=small_rp, col=small_col, src=0)
    assert small["stats"]["peak_slots"] < peak - 1
    with Ctx(peak - 1, **cfg) as ctx:
        status, _ = bfs_gpu(ctx, row_ptr, col, 0)
        assert status == T.TREES_ERR_CAPACITY
        status, level = bfs_gpu(ctx, small_rp, small_col, 0)  # the next job on the same context
        assert status == T.TREES_OK and np.array_equal(level, small["level"])
    with Ctx(peak, **cfg) as ctx:
        status, level = bfs_gpu(ctx, row_ptr, col, 0)
        assert status == T.TREES_OK
        assert np.array_equal(level, sim["level"])
        assert T.trees_stats(ctx)["peak_slots"] == peak
        check_trace(ctx, sim)


@pytest.mark.parametrize("tpt", [1, 4])
def test_all_programs_tasks_per_thread(tpt):
    cfg = dict(tasks_per_thread=tpt, block_size=256, trace=1)
    sim = oracle.tvm_run(oracle.NQUEENS, nq_n=9)
    with Ctx(1 << 16, **cfg) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_NQUEENS, n=9)) == T.TREES_OK
        assert T.trees_result(ctx, 0) == 352
        check_trace(ctx, sim)
    keys = gen.keys_u32(9, 300000)
    sim = oracle.tvm_run(oracle.MERGESORT, keys=keys, leaf=100)
    d = dev_u32(keys)
    with Ctx(1 << 16, **cfg) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_MERGESORT, n=keys.size, keys=d, leaf=100)) == T.TREES_OK
        assert np.array_equal(host_u32(d), sim["keys"])
        check_trace(ctx, sim, TRACE_FIELDS + ("maps",))
    row_ptr, col, _ = gen.rmat(14, 16, seed=3)
    sim = oracle.tvm_run(oracle.BFS, row_ptr=row_ptr, col=col, src=0)
    with Ctx(1 << 15, **cfg) as ctx:
        status, level = bfs_gpu(ctx, row_ptr, col, 0)
        assert status == T.TREES_OK and np.array_equal(level, sim["level"])
        check_trace(ctx, sim)


# ------------------------------------------------------------------ traversal (Fig. 2-4)

@pytest.mark.parametrize("sched", SCHEDS)
def test_fig3_postorder_exact(sched):
    left = np.array([1, 3, 5, -1, -1, -1], np.int32)
    right = np.array([2, 4, -1, -1, -1, -1], np.int32)
    sim = oracle.tvm_run(oracle.POSTORDER, left=left, right=right)
    l, r = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    ve = torch.empty(6, dtype=torch.int32, device="cuda")
    with Ctx(64, scheduler=sched, trace=1) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_POSTORDER, n=6, left=l, right=r, visit_epoch=ve)) == T.TREES_OK
        check_trace(ctx, sim)
        assert np.array_equal(ve.cpu().numpy(), sim["visit_epoch"])
        assert T.trees_stats(ctx)["final_slots"] == 0


@pytest.mark.parametrize("prog", [T.TREES_PROG_POSTORDER, T.TREES_PROG_PREORDER])
@pytest.mark.parametrize("nn", [1, 2, 1000, 50000])
def test_traversal_random(prog, nn):
    left, right = gen.binary_tree(nn, nn)
    sim = oracle.tvm_run(oracle.POSTORDER if prog == T.TREES_PROG_POSTORDER else oracle.PREORDER,
                         left=left, right=right)
    l, r = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    ve = torch.empty(nn, dtype=torch.int32, device="cuda")
    with Ctx(4 * nn + 8, trace=1) as ctx:
        assert run(ctx, T.make_job(prog, n=nn, left=l, right=r, visit_epoch=ve)) == T.TREES_OK
        assert np.array_equal(ve.cpu().numpy(), sim["visit_epoch"])
        check_trace(ctx, sim)


# ------------------------------------------------------------------ failures return status, never hang

def test_capacity_overflow_is_an_error_then_context_recovers():
    with Ctx(1000) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_FIB, n=20)) == T.TREES_ERR_CAPACITY
        assert run(ctx, T.make_job(T.TREES_PROG_FIB, n=10)) == T.TREES_OK
        assert T.trees_result(ctx, 0) == 55


@pytest.mark.parametrize("sched", SCHEDS)
def test_epoch_limit(sched):
    with Ctx(1 << 16, scheduler=sched, max_epochs=10) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_FIB, n=20)) == T.TREES_ERR_EPOCH_LIMIT


def test_map_capacity_overflow():
    keys = gen.keys_u32(5, 1 << 16)
    d = dev_u32(keys)
    with Ctx(1 << 16, map_capacity=8) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_MERGESORT, n=keys.size, keys=d)) == T.TREES_ERR_CAPACITY


def test_barrier_timeout_when_a_block_never_arrives():
    # the last block leaves in epoch 3 without arriving; every other block's
    # wait runs out after 50 ms and the run reports TIMEOUT
    with Ctx(1 << 16, inject_stall_epoch=3, timeout_ns=50_000_000) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_FIB, n=20)) == T.TREES_ERR_TIMEOUT
    with Ctx(1 << 16) as ctx:
        assert run(ctx, T.make_job(T.TREES_PROG_FIB, n=20)) == T.TREES_OK
        assert T.trees_result(ctx, 0) == 6765


def test_invalid_arguments_rejected_before_launch():
    with Ctx(1 << 10) as ctx:
        with pytest.raises(T.TreesError) as ei:
            T.trees_run(ctx, T.make_job(T.TREES_PROG_NQUEENS, n=17))
        assert ei.value.code == T.TREES_ERR_INVALID_ARG
        with pytest.raises(T.TreesError):
            T.trees_run(ctx, T.make_job(T.TREES_PROG_FIB, n=30, cutoff=31))
        with pytest.raises(T.TreesError):
            T.trees_run(ctx, T.make_job(99))


def test_create_on_caller_buffer():
    nbytes = T.trees_bytes_for(1 << 16, T.trees_default_config())
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    ctx = T.trees_create_on(buf, nbytes)
    try:
        assert T.trees_capacity(ctx) >= (1 << 16) - 64
        assert run(ctx, T.make_job(T.TREES_PROG_FIB, n=20)) == T.TREES_OK
        assert T.trees_result(ctx, 0) == 6765
    finally:
        T.trees_destroy(ctx)


def test_barrier_floor_positive():
    with Ctx(1 << 10) as ctx:
        us = T.trees_barrier_floor(ctx, 2000)
        assert 0.0 < us < 100.0
