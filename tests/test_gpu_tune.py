"""The autotuner picks the fastest candidate and caches it (GPU)."""
import json

import pytest
import torch

import paper_1608_00571_b300 as T

pytestmark = pytest.mark.gpu


def test_autotune_picks_fastest_and_caches(tmp_path):
    cache = tmp_path / "tune.json"
    job = T.make_job(T.TREES_PROG_FIB, n=22)
    best, ms, cands = T.trees_autotune(job, 1 << 18, reps=2, cache_path=str(cache), key="fib:n=22")
    assert len(cands) == 24 and all(c["status"] == T.TREES_OK for c in cands)
    assert ms == min(c["ms"] for c in cands)
    win = [c for c in cands if c["ms"] == ms][0]
    assert (best.block_size, best.tasks_per_thread, best.scheduler) == \
        (win["block_size"], win["tasks_per_thread"], win["scheduler"])
    d = json.loads(cache.read_text())
    assert d["fib:n=22"]["block_size"] == best.block_size
    # the tuned configuration runs the job correctly
    ctx = T.trees_create(1 << 18, best)
    try:
        T.trees_run(ctx, job, torch.cuda.current_stream())
        assert T.trees_sync(ctx) == T.TREES_OK and T.trees_result(ctx, 0) == 17711
    finally:
        T.trees_destroy(ctx)
    best2, ms2, cands2 = T.trees_autotune(job, 1 << 18, cache_path=str(cache), key="fib:n=22")
    assert cands2 == [] and best2.block_size == best.block_size and ms2 == pytest.approx(ms, rel=1e-4)


def test_autotune_restores_mergesort_keys():
    import numpy as np
    from paper_1608_00571_b300 import gen
    keys = gen.keys_u32(5, 100000)
    d = torch.from_numpy(keys.view(np.int32)).cuda()
    sc = torch.empty_like(d)
    job = T.make_job(T.TREES_PROG_MERGESORT, n=keys.size, keys=d, scratch=sc)
    best, ms, cands = T.trees_autotune(job, 1 << 12, reps=1)
    assert ms > 0 and len(cands) == 24
    assert all(c["status"] == T.TREES_OK for c in cands), [c for c in cands if c["status"]]
    assert np.array_equal(d.cpu().numpy().view(np.uint32), keys)   # the caller's keys are left as they were
