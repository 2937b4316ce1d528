"""The multi-rank path of bench.py on CPU: two gloo ranks, as torchrun would
start them (replicas only: the only collective is the max of the timed
region)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.reduce_max_ms(times[rank], dist, "cpu")
    q.put((rank, m, bench.job_value(world, 5, 1000, m), bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_whole_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [10.0, 14.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v, env in out:
        assert m == 14.0                                   # the slowest rank's timed region
        assert v == pytest.approx(2 * 5 * 1000 / 0.014)   # all ranks' work over that time
        assert env == (rank, 2, rank)


def test_single_rank_defaults():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_ms(3.5, None, "cpu") == 3.5
    assert bench.job_value(1, 2, 100, 1.0) == pytest.approx(200000.0)


def test_reference_arm_silent_on_other_ranks(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 0
    bench.run_reference(A(), 1, 2)      # rank 1 of 2: no work, no line
    assert capsys.readouterr().out == ""
