"""The checks bench.py applies to its full-size GPU results, on the CPU:
each accepts the oracle's answer and rejects plausible wrong ones."""
import numpy as np

import bench
import oracle
from paper_1608_00571_b300 import gen
from test_oracle import weighted_random_graph


def test_bfs_certificate():
    row_ptr, col, _ = gen.rmat(11, 16, seed=4)
    level, _ = oracle.bfs(row_ptr, col, 0)
    assert bench.bfs_certificate(row_ptr, col, 0, level)
    deep = np.where(level >= 2)[0][0]
    for bad in (level + (np.arange(level.size) == deep), np.where(np.arange(level.size) == deep, -1, level),
                np.where(level == 1, 2, level), np.where(np.arange(level.size) == 0, 1, level)):
        assert not bench.bfs_certificate(row_ptr, col, 0, bad.astype(np.int32))


def test_sssp_certificate():
    row_ptr, col, w = weighted_random_graph(200, 0.03, 6, 50, False)
    dist, _ = oracle.sssp_dijkstra(row_ptr, col, w, 0)
    level, _ = oracle.bfs(row_ptr, col, 0)
    assert bench.sssp_certificate(row_ptr, col, w, 0, dist, level)
    v = int(np.where((dist != oracle.SSSP_INF) & (dist > 0))[0][0])
    for delta in (1, -1):
        bad = dist.copy()
        bad[v] = np.uint64(int(bad[v]) + delta)
        assert not bench.sssp_certificate(row_ptr, col, w, 0, bad, level)


def test_dft_samples_match_the_definition():
    x = gen.signal(3, 1000).astype(np.complex128)
    ks = [0, 1, 333, 999]
    assert np.abs(bench.dft_samples(x, ks) - oracle.dft_at(x, ks)).max() < 1e-9


def test_fft_alg_bytes_and_host_cpu():
    assert bench.fft_alg_bytes(1 << 24, 16) == (16 * (1 << 24) * 21, 20)
    assert bench.fft_alg_bytes(16, 16) == (16 * 16, 0)
    h = bench.host_cpu()
    assert h["nproc"] >= 1 and "cpu_model" in h


def test_nqueens_table_matches_the_oracle():
    for n, count in bench.NQUEENS_SOLUTIONS.items():
        assert oracle.nqueens(n)[0] == count


def test_cpu_baseline_times_the_plain_recursion():
    cb = bench.cpu_baseline(0.2, bench.FIB34_TASKS)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["unit"] == "tasks/s"
    assert abs(cb["value"] - cb["fib34_jobs_per_s"] * bench.FIB34_TASKS) <= 1e-6 * cb["value"]
    assert cb["fib34_calls_per_s"] == cb["fib34_jobs_per_s"] * 18454929
    assert cb["tvm_simulator"]["value"] > 0
    assert bench.FIB34_TASKS == sum(oracle.fib_task_counts(34))


def test_reference_arm_prints_one_line_on_rank_0(capsys):
    import json

    class A:
        steps, warmup = 2, 1
    bench.run_reference(A(), 0, 1)
    lines = [x for x in capsys.readouterr().out.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "tasks/s" and d["steps"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
