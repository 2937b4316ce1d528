"""SSSP as tasks (Sec. 6.3) on the GPU against the oracle.

Shortest distances are unique, so they are compared exactly with Dijkstra.
Which thread shortens a distance first, and so how many relax tasks and
epochs a run takes, depends on the order of the races; those counts are
checked through properties that hold for any order.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1608_00571_b300 as T
from paper_1608_00571_b300 import gen
from test_oracle import weighted_random_graph

pytestmark = pytest.mark.gpu

SCHEDS = [T.TREES_SCHED_PERSISTENT, T.TREES_SCHED_GRAPH, T.TREES_SCHED_HOSTLOOP]


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).cuda()


def run_sssp(row_ptr, col, weight, src, cap, **cfg):
    nv = row_ptr.shape[0] - 1
    rp, cl = dev(row_ptr, np.int32), dev(col if col.size else np.zeros(1, np.int32), np.int32)
    w = dev(weight.view(np.int32) if weight.size else np.zeros(1, np.int32), np.int32)
    dist = torch.empty(nv, dtype=torch.int64, device="cuda")
    sched = torch.empty(nv, dtype=torch.int32, device="cuda")
    ctx = T.trees_create(cap, T.trees_default_config(trace=1, **cfg))
    try:
        T.trees_run(ctx, T.make_job(T.TREES_PROG_SSSP, n=src, row_ptr=rp, col=cl, weight=w, nv=nv, dist=dist,
                                    sched=sched), torch.cuda.current_stream())
        status = T.trees_sync(ctx)
        stats = T.trees_stats(ctx)
        trace = T.trees_trace(ctx)
    finally:
        T.trees_destroy(ctx)
    return status, dist.cpu().numpy().view(np.uint64), stats, trace


def check_counts(row_ptr, col, src, dist, stats, trace):
    reached = int((dist != oracle.SSSP_INF).sum())
    level, _ = oracle.bfs(row_ptr, col, src)
    assert stats["tasks"] >= reached                    # every reached vertex relaxed at least once
    assert stats["epochs"] >= int(level.max()) + 1      # a vertex L hops away is first forked in epoch >= L
    assert stats["joins"] == 0
    assert len(trace) == stats["epochs"]
    assert stats["final_slots"] == trace[-1]["lo"]      # no joins: only the last range is given back (Sec. 5.3)
    assert sum(t["valid"] for t in trace) == stats["tasks"]
    for i, t in enumerate(trace):
        assert t["cen"] == i and t["valid"] == t["hi"] - t["lo"]   # every forked relax task runs
        if i + 1 < len(trace):
            assert trace[i + 1]["hi"] - trace[i + 1]["lo"] == t["forks"]


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("nv,p,seed,wmax,directed", [(1, 0.0, 0, 5, False), (6, 0.0, 1, 5, True),
                                                     (12, 0.25, 2, 9, True), (40, 0.08, 3, 100, False),
                                                     (64, 0.05, 4, 1, True), (300, 0.02, 5, 1000, False)])
def test_sssp_random_graphs(sched, nv, p, seed, wmax, directed):
    row_ptr, col, weight = weighted_random_graph(nv, p, seed, wmax, directed)
    for src in {0, nv - 1}:
        want, _ = oracle.sssp_dijkstra(row_ptr, col, weight, src)
        status, dist, stats, trace = run_sssp(row_ptr, col, weight, src, 64 * nv + 64, scheduler=sched)
        assert status == T.TREES_OK
        assert np.array_equal(dist, want)
        check_counts(row_ptr, col, src, dist, stats, trace)


@pytest.mark.parametrize("bs,tpt", [(128, 4), (256, 1), (256, 2), (512, 2), (1024, 1)])
@pytest.mark.parametrize("scale", [10, 14])
def test_sssp_rmat_block_sizes(bs, tpt, scale):
    row_ptr, col, info = gen.rmat(scale, 16, seed=2)
    weight = gen.weights(3, row_ptr, col)
    want, _ = oracle.sssp_dijkstra(row_ptr, col, weight, 0)
    status, dist, stats, trace = run_sssp(row_ptr, col, weight, 0, 16 * info["nv"], block_size=bs,
                                          tasks_per_thread=tpt)
    assert status == T.TREES_OK
    assert np.array_equal(dist, want)
    check_counts(row_ptr, col, 0, dist, stats, trace)


@pytest.mark.parametrize("bs,tpt,grid", [(512, 1, 2), (512, 2, 3), (1024, 1, 2), (512, 1, 0)])
def test_sssp_claim_buffer_flushes_and_capacity(bs, tpt, grid):
    """The shapes with claim buffers (the shortened neighbours wait in a block part's buffer; its
    flush takes the atomic maxima that decide the forks): on two or three grid blocks every part
    flushes many times an epoch. Distances equal Dijkstra's, and a task vector far too small is a
    capacity error."""
    row_ptr, col, info = gen.rmat(14, 16, seed=4)
    weight = gen.weights(5, row_ptr, col)
    want, _ = oracle.sssp_dijkstra(row_ptr, col, weight, 0)
    cfg = dict(block_size=bs, tasks_per_thread=tpt)
    if grid:
        cfg["grid_blocks"] = grid
    status, dist, stats, trace = run_sssp(row_ptr, col, weight, 0, 16 * info["nv"], **cfg)
    assert status == T.TREES_OK
    assert np.array_equal(dist, want)
    check_counts(row_ptr, col, 0, dist, stats, trace)
    status, _, _, _ = run_sssp(row_ptr, col, weight, 0, info["nv"] // 4, **cfg)
    assert status == T.TREES_ERR_CAPACITY


def test_sssp_unit_weights_equal_gpu_bfs_levels():
    row_ptr, col, info = gen.rmat(13, 8, seed=7)
    nv = info["nv"]
    status, dist, stats, _ = run_sssp(row_ptr, col, np.ones(col.shape[0], np.uint32), 3, 4 * nv)
    assert status == T.TREES_OK
    level = torch.empty(nv, dtype=torch.int32, device="cuda")
    ctx = T.trees_create(nv + 64)
    try:
        T.trees_bfs(ctx, dev(row_ptr, np.int32), dev(col, np.int32), nv, 3, level, torch.cuda.current_stream())
        assert T.trees_sync(ctx) == T.TREES_OK
    finally:
        T.trees_destroy(ctx)
    lv = level.cpu().numpy()
    want = np.maximum(lv, 0).astype(np.uint64)
    want[lv < 0] = oracle.SSSP_INF
    assert np.array_equal(dist, want)
    # with unit weights a shortened vertex is never shortened again: one relax task per vertex
    assert stats["tasks"] == int((lv >= 0).sum()) and stats["epochs"] == int(lv.max()) + 1


def test_sssp_convenience_entry_point():
    row_ptr, col, info = gen.rmat(9, 16, seed=4)
    weight = gen.weights(5, row_ptr, col, wmax=1000)
    nv = info["nv"]
    want, _ = oracle.sssp_dijkstra(row_ptr, col, weight, 7)
    dist = torch.empty(nv, dtype=torch.int64, device="cuda")
    sched = torch.empty(nv, dtype=torch.int32, device="cuda")
    ctx = T.trees_create(16 * nv)
    try:
        T.trees_sssp(ctx, dev(row_ptr, np.int32), dev(col, np.int32), dev(weight.view(np.int32), np.int32), nv, 7,
                     dist, sched, torch.cuda.current_stream())
        assert T.trees_sync(ctx) == T.TREES_OK
    finally:
        T.trees_destroy(ctx)
    assert np.array_equal(dist.cpu().numpy().view(np.uint64), want)


def test_sssp_capacity_and_invalid_arguments():
    row_ptr, col, info = gen.rmat(10, 16, seed=2)
    weight = gen.weights(3, row_ptr, col)
    status, _, _, _ = run_sssp(row_ptr, col, weight, 0, 64)   # far fewer slots than relax tasks
    assert status == T.TREES_ERR_CAPACITY
    nv = info["nv"]
    rp, cl = dev(row_ptr, np.int32), dev(col, np.int32)
    dist = torch.empty(nv, dtype=torch.int64, device="cuda")
    sched = torch.empty(nv, dtype=torch.int32, device="cuda")
    ctx = T.trees_create(1024)
    try:
        for job in (T.make_job(T.TREES_PROG_SSSP, n=0, row_ptr=rp, col=cl, nv=nv, dist=dist, sched=sched),
                    T.make_job(T.TREES_PROG_SSSP, n=nv, row_ptr=rp, col=cl, weight=cl, nv=nv, dist=dist,
                               sched=sched)):
            with pytest.raises(T.TreesError) as ei:
                T.trees_run(ctx, job)
            assert ei.value.code == T.TREES_ERR_INVALID_ARG
    finally:
        T.trees_destroy(ctx)
