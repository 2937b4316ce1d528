"""The allocation-free fib entry point (trees_fib_noalloc) against the CPU
oracle's recursive Fibonacci and the regular entry point (trees_run on a
context), through the C ABI.

Callers that cannot allocate device memory while they run -- stream
captures that must not allocate, hosts with a fixed GPU memory budget,
plug-ins that do not own the allocator -- use trees_fib_noalloc, whose task
vector lives in a static device array inside the library.  This file is
collected last so that a failure here never hides the other tests.
"""
import pytest
import torch

import oracle
import paper_1608_00571_b300 as T

pytestmark = pytest.mark.gpu


def regular_fib(n, cutoff):
    ctx = T.trees_create(1 << 21, T.trees_default_config())
    try:
        T.trees_run(ctx, T.make_job(T.TREES_PROG_FIB, n=n, cutoff=cutoff), torch.cuda.current_stream())
        assert T.trees_sync(ctx) == T.TREES_OK
        return T.trees_result(ctx, 0)
    finally:
        T.trees_destroy(ctx)


def noalloc_fib(n, cutoff, out, status, stream):
    out.fill_(-1)
    status.fill_(-1)
    assert T.trees_fib_noalloc(n, cutoff, out, status, stream) == T.TREES_OK
    torch.cuda.synchronize()
    assert int(status.item()) == T.TREES_OK
    return int(out.item())


def test_noalloc_matches_oracle_and_regular_entry_point_twice_in_a_row():
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for n, cutoff in ((27, 0), (28, 12)):  # two calls in a row share the static array
        got = noalloc_fib(n, cutoff, out, status, stream)
        assert got == oracle.fib(n)[0] == regular_fib(n, cutoff)
    # the same job twice in a row gives the same answer (state left by the previous call is cleared)
    for _ in range(2):
        assert noalloc_fib(25, 0, out, status, stream) == oracle.fib(25)[0] == regular_fib(25, 0) == 75025


def test_noalloc_capacity_edge():
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # fib(28) with no cutoff peaks at 2F(29) - 1 = 1,028,457 of the 1,048,576 static slots
    assert noalloc_fib(28, 0, out, status, stream) == oracle.fib(28)[0] == 317811
    assert T.trees_fib_noalloc(29, 0, out, status, stream) == T.TREES_ERR_CAPACITY  # 2F(30) - 1 > 2^20
    assert noalloc_fib(34, 12, out, status, stream) == oracle.fib(34)[0] == 5702887  # 92,735 slots fit
    assert T.trees_fib_noalloc(20, 0, None, status, stream) == T.TREES_ERR_INVALID_ARG
