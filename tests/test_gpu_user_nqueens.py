"""A second user task program through the SDK: N-Queens solution counting
(paper_1608_00571_b300/examples/nqueens.cu), with a variable number of
children per task (one per safe column) and a join that adds their counts.
It is compiled with the public include directory alone on the include path,
run by trees_run, and compared exactly with the oracle: the solution count
with the backtracking recursion, and the task counts and the whole
per-epoch trace with the TVM simulator's built-in N-Queens program (the same
task tree under other type numbers)."""
import ctypes
import os

import pytest
import torch

import oracle
import paper_1608_00571_b300 as T
from paper_1608_00571_b300 import build as tbuild

pytestmark = pytest.mark.gpu

EXAMPLES = os.path.join(os.path.dirname(os.path.abspath(T.__file__)), "examples")
TRACE_FIELDS = ("cen", "lo", "hi", "valid", "forks", "joined")


@pytest.fixture(scope="module")
def program():
    so = tbuild.build_program(os.path.join(EXAMPLES, "nqueens.cu"), os.path.join(EXAMPLES, "libnqueens.so"))
    return ctypes.CDLL(so).trees_nqueens_program


def run_nq(program, n, **cfg):
    ctx = T.trees_create(1 << 20, T.trees_default_config(trace=1, map_capacity=1, **cfg))
    try:
        job = T.make_job(T.TREES_PROG_USER, user_program=program, user_type=1, user_a0=0, user_a1=0,
                         user_val=(n,))
        T.trees_run(ctx, job, torch.cuda.current_stream())
        status = T.trees_sync(ctx)
        return status, T.trees_result(ctx, 0), T.trees_stats(ctx), T.trees_trace(ctx)
    finally:
        T.trees_destroy(ctx)


@pytest.mark.parametrize("n", list(range(1, 12)))
def test_user_nqueens_against_oracle(program, n):
    status, result, stats, trace = run_nq(program, n)
    assert status == T.TREES_OK
    sols, rows, joins = oracle.nqueens(n)
    assert result == sols
    sim = oracle.tvm_run(oracle.NQUEENS, nq_n=n)
    assert sim["stats"]["root_result"] == sols
    assert (stats["tasks"], stats["joins"]) == (rows + joins, joins)
    if n >= 4:  # the tree reaches row n: n forward epochs, n - 1 join epochs and the root's join
        assert stats["epochs"] == 2 * n + 1
    for k in ("epochs", "tasks", "forks", "joins", "peak_slots", "final_slots"):
        assert stats[k] == sim["stats"][k], k
    assert len(trace) == len(sim["trace"])
    for i, (g, o) in enumerate(zip(trace, sim["trace"])):
        for f in TRACE_FIELDS:
            assert g[f] == int(o[f]), (i, f, g, o)


@pytest.mark.parametrize("bs,tpt", [(128, 1), (256, 4), (512, 2), (1024, 1)])
@pytest.mark.parametrize("grid", [0, 2])
def test_user_nqueens_block_shapes(program, bs, tpt, grid):
    status, result, stats, trace = run_nq(program, 10, block_size=bs, tasks_per_thread=tpt, grid_blocks=grid)
    assert status == T.TREES_OK and result == 724
    sim = oracle.tvm_run(oracle.NQUEENS, nq_n=10)
    assert [(t["lo"], t["hi"], t["valid"], t["forks"]) for t in trace] == \
        [(int(o["lo"]), int(o["hi"]), int(o["valid"]), int(o["forks"])) for o in sim["trace"]]
