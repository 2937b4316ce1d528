"""A user task program (include/trees_program.cuh) through the C ABI.

The chunked-sum example (paper_1608_00571_b300/examples/chunk_sum.cu: arity-k forks,
a join that adds its children, a block-cooperative map per leaf) is compiled
into its own library and run by trees_run.  Integer work, so everything is
exact: the sum against numpy's uint64 sum, and the counts and the whole
per-epoch trace against the oracle's model of the task tree."""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
import paper_1608_00571_b300 as T
from paper_1608_00571_b300 import build as tbuild
from paper_1608_00571_b300 import gen

pytestmark = pytest.mark.gpu

EXAMPLES = os.path.join(os.path.dirname(os.path.abspath(T.__file__)), "examples")
TRACE_FIELDS = ("cen", "lo", "hi", "valid", "forks", "joined", "maps")


@pytest.fixture(scope="module")
def program():
    so = tbuild.build_program(os.path.join(EXAMPLES, "chunk_sum.cu"),
                              os.path.join(EXAMPLES, "libchunk_sum.so"))
    lib = ctypes.CDLL(so)
    return lib.trees_chunk_sum


def run_sum(program, keys, chunk, arity, cap=None, upk=0, **cfg):
    n = keys.shape[0]
    d = torch.from_numpy(keys.view(np.int32)).cuda() if n else torch.zeros(1, dtype=torch.int32, device="cuda")
    st_model, _ = oracle.chunk_sum_tree(n, chunk, arity)
    ctx = T.trees_create(cap or st_model["peak_slots"] + 64, T.trees_default_config(trace=1, **cfg))
    try:
        job = T.make_job(T.TREES_PROG_USER, user_program=program, user_type=1, user_a0=0, user_a1=n,
                         user_ptr=(d,), user_val=(chunk, arity, upk))
        T.trees_run(ctx, job, torch.cuda.current_stream())
        status = T.trees_sync(ctx)
        stats = T.trees_stats(ctx)
        trace = T.trees_trace(ctx)
        result = T.trees_result(ctx, 0)
    finally:
        T.trees_destroy(ctx)
    return status, result, stats, trace


@pytest.mark.parametrize("n,chunk,arity", [(0, 4096, 8), (1, 4096, 8), (4096, 4096, 8), (4097, 4096, 8),
                                           (100_000, 1000, 3), (1 << 20, 4096, 8), (123_457, 7, 16),
                                           (3_000_001, 4096, 2)])
def test_chunk_sum_against_oracle(program, n, chunk, arity):
    keys = gen.keys_u32(n + 3, n)
    status, result, stats, trace = run_sum(program, keys, chunk, arity)
    assert status == T.TREES_OK
    assert result == int(keys.astype(np.uint64).sum())
    st, tr = oracle.chunk_sum_tree(n, chunk, arity)
    for f in ("epochs", "tasks", "joins", "maps", "peak_slots", "final_slots"):
        assert stats[f] == st[f], f
    assert len(trace) == len(tr)
    for i, (g, o) in enumerate(zip(trace, tr)):
        for f in TRACE_FIELDS:
            assert g[f] == o[f], (i, f, g, o)


@pytest.mark.parametrize("n,chunk,arity,upk", [(1 << 20, 4096, 8, 1000), (100_000, 1000, 3, 7), (123_457, 7, 16, 2),
                                                (4097, 4096, 8, 4096), (50_000, 50_000, 2, 333)])
def test_chunk_sum_multi_unit_maps(program, n, chunk, arity, upk):
    """Leaves emit 0 and map ceil(len / upk) units that add their partial sums:
    maps of many units, each unit's index, and an emit together with a map."""
    keys = gen.keys_u32(n + 11, n)
    # map units count against the map capacity (default: the task-vector capacity)
    status, result, stats, trace = run_sum(program, keys, chunk, arity, upk=upk, map_capacity=n // upk + 1024)
    assert status == T.TREES_OK
    assert result == int(keys.astype(np.uint64).sum())
    st, tr = oracle.chunk_sum_tree(n, chunk, arity)
    assert (stats["maps"], stats["epochs"], stats["tasks"]) == (st["maps"], st["epochs"], st["tasks"])
    assert [t["maps"] for t in trace] == [t["maps"] for t in tr]


@pytest.mark.parametrize("bs,tpt", [(128, 1), (256, 4), (512, 2), (1024, 1)])
def test_chunk_sum_block_shapes(program, bs, tpt):
    n = 777_777
    keys = gen.keys_u32(5, n)
    status, result, stats, _ = run_sum(program, keys, 512, 5, block_size=bs, tasks_per_thread=tpt)
    assert status == T.TREES_OK and result == int(keys.astype(np.uint64).sum())
    assert stats["maps"] == oracle.chunk_sum_tree(n, 512, 5)[0]["maps"]


def test_user_program_errors(program):
    keys = gen.keys_u32(1, 50_000)
    status, _, _, _ = run_sum(program, keys, 16, 4, cap=32)  # far fewer slots than tasks
    assert status == T.TREES_ERR_CAPACITY
    status, _, _, _ = run_sum(program, keys, 4096, 8, upk=10, map_capacity=64)  # more map units than map capacity
    assert status == T.TREES_ERR_CAPACITY
    d = torch.from_numpy(keys.view(np.int32)).cuda()
    for cfg, kw in [({}, dict(user_program=None, user_type=1)), ({}, dict(user_program=program, user_type=0)),
                    ({}, dict(user_program=program, user_type=T.TREES_NUM_TASK_TYPES + 1)),
                    ({"scheduler": T.TREES_SCHED_GRAPH}, dict(user_program=program, user_type=1)),
                    ({"scheduler": T.TREES_SCHED_HOSTLOOP}, dict(user_program=program, user_type=1))]:
        ctx = T.trees_create(1024, T.trees_default_config(**cfg))
        try:
            with pytest.raises(T.TreesError) as ei:
                T.trees_run(ctx, T.make_job(T.TREES_PROG_USER, user_a1=keys.size, user_ptr=(d,), user_val=(16, 4),
                                            **kw))
            assert ei.value.code == T.TREES_ERR_INVALID_ARG
        finally:
            T.trees_destroy(ctx)
