"""Batched and served task trees against each job's solo oracle run.

Every job of a batch (or of the server's mix) must give exactly what it
gives alone: the root result, its epoch count, its task and join counts, and
for mergesort the sorted keys.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1608_00571_b300 as T
from paper_1608_00571_b300 import gen

pytestmark = pytest.mark.gpu


def fib_closed(n):
    a, b = 0, 1
    for _ in range(n):
        a, b = b, a + b
    return a


class Mix:
    """A small deterministic job mix with its oracle expectations."""

    def __init__(self, njobs, seed=0, sort_sizes=(1000, 1024, 3000, 4097, 20000, 70000)):
        self.jobs, self.expect, self.keys, self.bufs = [], [], {}, []
        for i in range(njobs):
            kind = (i + seed) % 4
            if kind == 0:
                n = 8 + (i * 7) % 13
                sim = oracle.tvm_run(oracle.FIB, fib_n=n)
                job = T.make_job(T.TREES_PROG_FIB, n=n)
            elif kind == 1:
                n = 4 + (i * 5) % 6
                sim = oracle.tvm_run(oracle.NQUEENS, nq_n=n)
                job = T.make_job(T.TREES_PROG_NQUEENS, n=n)
            elif kind == 2:
                n = sort_sizes[i % len(sort_sizes)]
                k = gen.keys_u32(1000 + i, n)
                sim = oracle.tvm_run(oracle.MERGESORT, keys=k)
                d = torch.from_numpy(k.view(np.int32)).cuda()
                sc = torch.empty_like(d)
                self.bufs += [d, sc]
                self.keys[i] = (d, sim["keys"])
                job = T.make_job(T.TREES_PROG_MERGESORT, n=n, keys=d, scratch=sc)
            else:
                n = 12 + (i * 3) % 9
                sim = oracle.tvm_run(oracle.FIB, fib_n=n, fib_cutoff=7)
                job = T.make_job(T.TREES_PROG_FIB, n=n, cutoff=7)
            self.jobs.append(job)
            self.expect.append(sim["stats"])

    def check(self, results, skip_status=()):
        for i, (r, e) in enumerate(zip(results, self.expect)):
            if i in skip_status:
                continue
            assert r["status"] == T.TREES_OK, (i, r)
            assert r["epochs"] == e["epochs"], (i, r, e)
            assert r["tasks"] == e["tasks"], (i, r, e)
            assert r["joins"] == e["joins"], (i, r, e)
            if self.jobs[i].program in (T.TREES_PROG_FIB, T.TREES_PROG_NQUEENS):
                assert r["result"] == e["root_result"], (i, r, e)
        for i, (d, want) in self.keys.items():
            if i in skip_status:
                continue
            assert np.array_equal(d.cpu().numpy().view(np.uint32), want), i


@pytest.mark.parametrize("bs", [128, 256, 512, 1024])
def test_batch_matches_solo_oracle(bs):
    mix = Mix(48)
    ctx = T.trees_create(1 << 22, T.trees_default_config(block_size=bs))
    try:
        T.trees_batch_run(ctx, mix.jobs, stream=torch.cuda.current_stream())
        status, res, steps = T.trees_batch_results(ctx, len(mix.jobs))
        assert status == T.TREES_OK
        mix.check(res)
        assert steps == max(e["epochs"] for e in mix.expect)   # one global step per epoch of the longest job
    finally:
        T.trees_destroy(ctx)


def test_batch_job_exceeding_its_segment_fails_alone():
    mix = Mix(12)
    segs = [T.trees_job_slots(j)[0] for j in mix.jobs]
    segs[0] = 10  # job 0 is fib(8): needs 67 slots
    ctx = T.trees_create(1 << 20)
    try:
        T.trees_batch_run(ctx, mix.jobs, segs)
        status, res, _ = T.trees_batch_results(ctx, len(mix.jobs))
        assert status == T.TREES_OK
        assert res[0]["status"] == T.TREES_ERR_CAPACITY
        mix.check(res, skip_status={0})
    finally:
        T.trees_destroy(ctx)


def test_job_slots_exact_and_estimate():
    for n in (2, 10, 20):
        slots, exact = T.trees_job_slots(T.make_job(T.TREES_PROG_FIB, n=n))
        assert exact and slots == oracle.tvm_run(oracle.FIB, fib_n=n)["stats"]["peak_slots"]
    for n in (1024, 5000, 1 << 16):
        slots, exact = T.trees_job_slots(T.make_job(T.TREES_PROG_MERGESORT, n=n, keys=1, scratch=1))
        assert exact and slots == oracle.tvm_run(oracle.MERGESORT, keys=gen.keys_u32(1, n))["stats"]["peak_slots"]
    slots, exact = T.trees_job_slots(T.make_job(T.TREES_PROG_NQUEENS, n=8))
    assert not exact and slots >= oracle.nqueens(8)[1]


def test_nqueens_estimate_overflow_then_retry():
    job = T.make_job(T.TREES_PROG_NQUEENS, n=12)
    est, exact = T.trees_job_slots(job)
    sols, rows, joins = oracle.nqueens(12)
    assert not exact and est < rows           # the estimate is too small for n = 12
    ctx = T.trees_create(8 * est)
    try:
        T.trees_batch_run(ctx, [job], [est])
        _, res, _ = T.trees_batch_results(ctx, 1)
        assert res[0]["status"] == T.TREES_ERR_CAPACITY
        T.trees_batch_run(ctx, [job], [4 * est])   # re-admitted with more memory
        _, res, _ = T.trees_batch_results(ctx, 1)
        assert res[0]["status"] == T.TREES_OK and res[0]["result"] == sols == 14200
        assert res[0]["tasks"] == rows + joins
    finally:
        T.trees_destroy(ctx)


def test_batch_rejects_bfs_and_oversubscription():
    ctx = T.trees_create(1000)
    try:
        with pytest.raises(T.TreesError) as ei:
            T.trees_batch_run(ctx, [T.make_job(T.TREES_PROG_BFS, n=0, row_ptr=1, col=1, level=1, nv=4)])
        assert ei.value.code == T.TREES_ERR_INVALID_ARG
        with pytest.raises(T.TreesError) as ei:
            T.trees_batch_run(ctx, [T.make_job(T.TREES_PROG_FIB, n=20)])   # needs 21,891 slots
        assert ei.value.code == T.TREES_ERR_ADMISSION
    finally:
        T.trees_destroy(ctx)


def test_server_admits_as_memory_frees():
    mix = Mix(40, seed=1)
    # a pool and a job table far smaller than the mix: jobs wait for entries and segments
    srv = T.trees_server_create(1 << 18, 6, 3, T.trees_default_config(block_size=512))
    try:
        ids = [T.trees_server_submit(srv, j) for j in mix.jobs]
        results = {}
        launches = 0
        while len(results) < len(ids):
            T.trees_server_step(srv, torch.cuda.current_stream())
            launches += 1
            for r in T.trees_server_poll(srv):
                results[r["id"]] = r
            assert launches < 10000
        q, run, L = T.trees_server_stats(srv)
        assert (q, run) == (0, 0) and L == launches
        mix.check([results[i] for i in ids])
    finally:
        T.trees_server_destroy(srv)


@pytest.mark.parametrize("plain", [False, True])
def test_server_replay_results_equal_alone_and_in_the_mix(plain):
    mix = Mix(36, seed=2)
    arrivals = gen.poisson_arrivals(43, len(mix.jobs), 3000.0)
    srv = T.trees_server_create(1 << 20, 16, 4)
    try:
        lat, res = T.trees_server_replay(srv, mix.jobs, arrivals, plain=plain, stream=torch.cuda.current_stream())
        assert all(x > 0 for x in lat)
        mix.check(res)
    finally:
        T.trees_server_destroy(srv)


def test_full_job_mix_4096():
    """The batched configuration at full size: 4096 jobs (seed 42) in one launch,
    checked against closed forms (fib), the oracle (N-Queens, and the first 64
    sorts) and, key for key, a sorted copy of every other sort's input."""
    kind, param, kseed = gen.jobs(42, 4096)
    jobs, keys = [], {}
    for i in range(4096):
        if kind[i] == gen.JOB_FIB:
            jobs.append(T.make_job(T.TREES_PROG_FIB, n=int(param[i])))
        elif kind[i] == gen.JOB_NQUEENS:
            jobs.append(T.make_job(T.TREES_PROG_NQUEENS, n=int(param[i])))
        else:
            k = gen.keys_u32(int(kseed[i]), int(param[i]))
            d = torch.from_numpy(k.view(np.int32)).cuda()
            sc = torch.empty_like(d)
            keys[i] = (d, sc, k)
            jobs.append(T.make_job(T.TREES_PROG_MERGESORT, n=int(param[i]), keys=d, scratch=sc))
    segs = [T.trees_job_slots(j)[0] for j in jobs]
    ctx = T.trees_create(sum(segs) + 1024, T.trees_default_config(map_capacity=1 << 22))
    try:
        T.trees_batch_run(ctx, jobs, segs, torch.cuda.current_stream())
        status, res, steps = T.trees_batch_results(ctx, 4096)
        assert status == T.TREES_OK
        nq_cache = {}
        for i, r in enumerate(res):
            assert r["status"] == T.TREES_OK, (i, r)
            if kind[i] == gen.JOB_FIB:
                n = int(param[i])
                assert r["result"] == fib_closed(n)
                assert r["epochs"] == 2 * n - 1 and r["tasks"] == 3 * fib_closed(n + 1) - 2
            elif kind[i] == gen.JOB_NQUEENS:
                n = int(param[i])
                sols, rows, joins = nq_cache.setdefault(n, oracle.nqueens(n))
                assert r["result"] == sols and r["tasks"] == rows + joins and r["epochs"] == 2 * n + 1
        for n_checked, (i, (d, sc, k)) in enumerate(keys.items()):
            if n_checked < 64:
                assert np.array_equal(d.cpu().numpy().view(np.uint32), oracle.mergesort(k)), i
            else:
                # every other sort against a sorted copy of its own input made on the device (torch.sort
                # of the keys as unsigned values: int64 keeps their order), key for key
                want = torch.sort(torch.from_numpy(k.astype(np.int64)).cuda()).values
                assert torch.equal(d.to(torch.int64) & 0xFFFFFFFF, want), i
    finally:
        T.trees_destroy(ctx)
