"""The FFT as tasks (Sec. 6.2, Fig. 6) on the GPU against the oracle.

The transform is floating point, so values are compared with the error bound
of radix-2 Cooley-Tukey in floating point (Higham, Accuracy and Stability of
Numerical Algorithms, 2nd ed., Thm. 24.2): with unit roundoff u and twiddles
within mu of exact, ||X_computed - X||_2 <= (L eta / (1 - L eta)) ||X||_2,
L = log2 N, eta = mu + gamma_4 (sqrt 2 + mu), gamma_4 = 4u / (1 - 4u).  Here
u = 2^-24 (fp32) and every twiddle component is within 1 ulp (<= 2u of a
value of modulus <= 1, sincospif), so mu <= 2u and eta < 8u.  The oracle is
fp64 (its own error is below 1e-12 relative).

Everything integer is exact: the task tree, the per-epoch trace and the map
counts equal the oracle's TVM run, and the output is bit-identical across
leaf sizes, cutoffs, block sizes and schedulers (every butterfly is one fixed
sequence of roundings wherever it runs).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1608_00571_b300 as T
from paper_1608_00571_b300 import gen

pytestmark = pytest.mark.gpu

SCHEDS = [T.TREES_SCHED_PERSISTENT, T.TREES_SCHED_GRAPH, T.TREES_SCHED_HOSTLOOP]
TRACE_FIELDS = ("cen", "lo", "hi", "valid", "forks", "joined", "maps")
U32 = 2.0 ** -24


def bound(n):
    """Relative 2-norm error bound of Thm. 24.2 for an n-point fp32 FFT, plus the oracle's own error."""
    lg = max(1, int(math.log2(n)))
    eta = 8 * U32
    return lg * eta / (1 - lg * eta) + 1e-12


def fft_gpu(x, leaf=0, cutoff=0, cap=None, **cfg):
    n = x.shape[0]
    xi = torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex64).view(np.float32)).cuda()
    xo = torch.full((2 * n,), float("nan"), dtype=torch.float32, device="cuda")
    slots, _ = T.trees_job_slots(T.make_job(T.TREES_PROG_FFT, n=n, leaf=leaf, cutoff=cutoff, fft_in=1, fft_out=1))
    ctx = T.trees_create(cap or slots, T.trees_default_config(trace=1, **cfg))
    try:
        T.trees_run(ctx, T.make_job(T.TREES_PROG_FFT, n=n, leaf=leaf, cutoff=cutoff, fft_in=xi, fft_out=xo),
                    torch.cuda.current_stream())
        status = T.trees_sync(ctx)
        stats = T.trees_stats(ctx)
        trace = T.trees_trace(ctx)
    finally:
        T.trees_destroy(ctx)
    assert torch.equal(xi.cpu(), torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex64).view(np.float32)))
    return status, xo.cpu().numpy().view(np.complex64), stats, trace


def check_close(got, want):
    assert np.all(np.isfinite(got.view(np.float32)))
    err = np.linalg.norm(got.astype(np.complex128) - want)
    assert err <= bound(want.shape[0]) * np.linalg.norm(want), (err, np.linalg.norm(want))


def check_tree(n, leaf, cutoff, stats, trace):
    sim = oracle.tvm_run(oracle.FFT, x=np.zeros(n), fft_leaf=leaf or 16, fft_cutoff=cutoff)
    for f in ("epochs", "tasks", "joins", "maps", "peak_slots", "final_slots"):
        assert stats[f] == sim["stats"][f], f
    assert len(trace) == len(sim["trace"])
    for i, (g, o) in enumerate(zip(trace, sim["trace"])):
        for f in TRACE_FIELDS:
            assert g[f] == int(o[f]), (i, f, g, o)


@pytest.mark.parametrize("lg", [0, 1, 2, 3, 4, 5, 7, 9, 11])
@pytest.mark.parametrize("leaf,cutoff", [(1, 0), (2, 1 << 30), (16, 0), (8, 64)])
def test_fft_small_against_definition(lg, leaf, cutoff):
    n = 1 << lg
    x = gen.signal(100 + lg, n)
    status, X, stats, trace = fft_gpu(x, leaf, cutoff)
    assert status == T.TREES_OK
    check_close(X, oracle.dft(x.astype(np.complex128)))
    check_tree(n, leaf, cutoff, stats, trace)


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("bs,tpt", [(128, 4), (256, 1), (256, 2), (512, 4), (1024, 2)])
def test_fft_schedulers_and_block_sizes(sched, bs, tpt):
    n = 1 << 14
    x = gen.signal(7, n)
    want = oracle.tvm_run(oracle.FFT, x=x.astype(np.complex128), fft_leaf=4, fft_cutoff=256)["X"]
    status, X, stats, trace = fft_gpu(x, 4, 256, scheduler=sched, block_size=bs, tasks_per_thread=tpt)
    assert status == T.TREES_OK
    check_close(X, want)
    check_tree(n, 4, 256, stats, trace)


def test_fft_bit_identical_across_configurations():
    n = 1 << 13
    x = gen.signal(9, n)
    outs = []
    for leaf, cutoff, sched, bs, tpt in [(16, 0, 0, 256, 2), (1, 0, 0, 256, 2), (2, 1 << 30, 0, 512, 1),
                                         (8, 32, 1, 128, 4), (4, 4096, 2, 1024, 1), (16, 8, 0, 1024, 4)]:
        status, X, _, _ = fft_gpu(x, leaf, cutoff, scheduler=sched, block_size=bs, tasks_per_thread=tpt)
        assert status == T.TREES_OK
        outs.append(X.view(np.uint32))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("lg", [14, 20])
def test_fft_leaf_epoch_buffers_every_block_size(lg):
    """The 16-point leaf epoch at every block size: its next slot's points in shared memory
    (256 threads), its outputs staged too (128 threads; 512 threads, in dynamic shared memory)
    or neither (1024 threads). 2^14 points leave most warps partly idle; 2^20 give every thread
    several slots, the last one partial. The outputs are bit-identical across shapes, within the
    radix-2 bound of the oracle's transform, and every epoch matches the oracle's task tree."""
    n = 1 << lg
    x = gen.signal(lg + 100, n)
    want = oracle.tvm_run(oracle.FFT, x=x.astype(np.complex128), fft_leaf=16, fft_cutoff=0)["X"] if lg <= 14 else None
    outs = []
    for bs, tpt in [(128, 1), (128, 2), (256, 1), (512, 1), (512, 2), (1024, 1)]:
        status, X, stats, trace = fft_gpu(x, 16, 0, block_size=bs, tasks_per_thread=tpt)
        assert status == T.TREES_OK, (bs, tpt)
        if want is not None:
            check_close(X, want)
            check_tree(n, 16, 0, stats, trace)
        else:
            assert stats["epochs"] == 2 * (lg - 4) + 1
        outs.append(X.view(np.uint32))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    if want is None:  # Parseval holds to the bound
        x64 = x.astype(np.complex128)
        norm_X = math.sqrt(n) * np.linalg.norm(x64)
        assert abs(np.linalg.norm(outs[0].view(np.complex64).astype(np.complex128)) - norm_X) <= bound(n) * norm_X


@pytest.mark.parametrize("lg", [16, 18])
def test_fft_mid_sizes_against_oracle_tvm(lg):
    n = 1 << lg
    x = gen.signal(lg, n)
    want = oracle.tvm_run(oracle.FFT, x=x.astype(np.complex128), fft_leaf=16, fft_cutoff=0)["X"]
    status, X, stats, trace = fft_gpu(x, 16, 64)
    assert status == T.TREES_OK
    check_close(X, want)
    check_tree(n, 16, 64, stats, trace)


@pytest.mark.parametrize("bs,tpt", [(256, 1), (512, 1), (512, 2)])
def test_fft_full_size_sampled_outputs(bs, tpt):
    """2^24 points in the benchmark's configuration, at the shapes the autotuner picks from: every
    output is finite, Parseval holds to the bound, and sampled outputs match the definition."""
    n, leaf, cutoff = 1 << 24, 16, 0
    x = gen.signal(1, n)
    status, X, stats, _ = fft_gpu(x, leaf, cutoff, block_size=bs, tasks_per_thread=tpt)
    assert status == T.TREES_OK
    assert stats["epochs"] == 2 * 20 + 1
    x64 = x.astype(np.complex128)
    norm_X = math.sqrt(n) * np.linalg.norm(x64)  # Parseval: ||X|| = sqrt(n) ||x||
    e = bound(n)
    assert abs(np.linalg.norm(X.astype(np.complex128)) - norm_X) <= e * norm_X
    rng = np.random.default_rng(0)
    ks = np.concatenate([[0, 1, n // 2, n - 1], rng.integers(0, n, 4)])
    want = oracle.dft_at(x64, ks)
    # a single output's error is at most the whole error vector's norm
    assert np.all(np.abs(X[ks].astype(np.complex128) - want) <= e * norm_X)


def test_fft_edge_cases_and_invalid_arguments():
    one = gen.signal(3, 1)
    status, X, stats, _ = fft_gpu(one)
    assert status == T.TREES_OK and X[0] == one[0] and stats["tasks"] == 1
    x = gen.signal(4, 64)
    status, _, _, _ = fft_gpu(x, 1, 0, cap=8)  # 127 task slots needed
    assert status == T.TREES_ERR_CAPACITY
    buf = torch.zeros(4 * 64 + 8, dtype=torch.float32, device="cuda")
    src, dst = buf[:128], buf[128:256]
    ctx = T.trees_create(1024)
    try:
        bad = [dict(n=48, fft_in=src, fft_out=dst), dict(n=0, fft_in=src, fft_out=dst),
               dict(n=64, leaf=32, fft_in=src, fft_out=dst), dict(n=64, leaf=3, fft_in=src, fft_out=dst),
               dict(n=64, fft_in=None, fft_out=dst), dict(n=64, fft_in=src, fft_out=None),
               dict(n=64, fft_in=src, fft_out=buf[64:192]),          # overlapping
               dict(n=64, fft_in=buf[1:129], fft_out=dst),           # 4-byte aligned only
               dict(n=1 << 26, fft_in=src, fft_out=dst)]             # above 2^25 points
        for kw in bad:
            with pytest.raises(T.TreesError) as ei:
                T.trees_run(ctx, T.make_job(T.TREES_PROG_FFT, **kw))
            assert ei.value.code == T.TREES_ERR_INVALID_ARG, kw
    finally:
        T.trees_destroy(ctx)


def test_fft_convenience_entry_point():
    n = 1 << 10
    x = gen.signal(21, n)
    xi = torch.from_numpy(x.view(np.float32)).cuda()
    xo = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    ctx = T.trees_create(4096)
    try:
        T.trees_fft(ctx, xi, xo, n, 8, 32, torch.cuda.current_stream())
        assert T.trees_sync(ctx) == T.TREES_OK
    finally:
        T.trees_destroy(ctx)
    check_close(xo.cpu().numpy().view(np.complex64), oracle.dft(x.astype(np.complex128)))
