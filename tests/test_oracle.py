"""Pins the CPU oracle to facts outside itself (CPU only).

Each check compares the oracle with something it does not compute the same
way: printed values from the paper's worked example (Sec. 5.3, golden file),
closed forms (Fibonacci identities), known counts (OEIS A000170), brute force
on tiny inputs (permutations, Floyd-Warshall), and library routines
(numpy sort, scipy shortest paths).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1608_00571_b300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fib_fast_doubling(n):
    """F(n) by the fast-doubling identities F(2k)=F(k)(2F(k+1)-F(k)),
    F(2k+1)=F(k)^2+F(k+1)^2 (a different algorithm from the oracle's)."""
    def fd(k):
        if k == 0:
            return 0, 1
        a, b = fd(k // 2)
        c = a * (2 * b - a)
        d = a * a + b * b
        return (d, c + d) if k % 2 else (c, d)
    return fd(n)[0]


def load_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    return rows


# ----------------------------------------------------------------- Fibonacci

@pytest.mark.parametrize("n", list(range(0, 28)))
def test_fib_value_and_calls(n):
    v, calls = oracle.fib(n)
    assert v == fib_fast_doubling(n)
    # the naive recursion makes 2F(n+1)-1 calls
    assert calls == 2 * fib_fast_doubling(n + 1) - 1


def test_fib_known_values():
    assert oracle.fib(20)[0] == 6765
    assert oracle.fib(34)[0] == 5702887


@pytest.mark.parametrize("n", [2, 3, 5, 10, 20, 25])
def test_fib_tvm_closed_forms(n):
    r = oracle.tvm_run(oracle.FIB, fib_n=n)
    st = r["stats"]
    F = fib_fast_doubling
    assert st["root_result"] == F(n)
    assert st["tasks"] == 3 * F(n + 1) - 2          # fib calls + one sum per internal call
    assert st["joins"] == F(n + 1) - 1
    assert st["peak_slots"] == 2 * F(n + 1) - 1     # nothing is reclaimed until the deepest level
    assert st["epochs"] == 2 * n - 1                # n forward levels, n-1 join levels (Sec. 4.4.1)
    assert st["final_slots"] == 0                   # TV and stacks empty together (Sec. 5.3)
    # the fib task tree's width at each depth (brute force on the tree) is the valid count
    # of the forward epochs
    level = [n]
    for d in range(n):
        assert r["trace"][d]["valid"] == len(level)
        assert r["trace"][d]["cen"] == d
        level = [c for x in level if x >= 2 for c in (x - 1, x - 2)]
    assert not level


@pytest.mark.parametrize("n", [0, 1])
def test_fib_tvm_leaf_root(n):
    st = oracle.tvm_run(oracle.FIB, fib_n=n)["stats"]
    assert (st["root_result"], st["tasks"], st["epochs"]) == (n, 1, 1)


@pytest.mark.parametrize("n,c", [(20, 12), (25, 12), (34, 12), (15, 14), (15, 15)])
def test_fib_cutoff_closed_forms(n, c):
    F = fib_fast_doubling
    r = oracle.tvm_run(oracle.FIB, fib_n=n, fib_cutoff=c)
    st = r["stats"]
    assert st["root_result"] == F(n)
    if n <= c:
        assert st["tasks"] == 1 and st["epochs"] == 1
        return
    # a subtree rooted at m has 2F(m-c+2)-1 calls when leaves are m <= c
    calls = 2 * F(n - c + 2) - 1
    assert st["tasks"] == calls + (F(n - c + 2) - 1)
    assert oracle.fib_task_counts(n, c) == (calls, F(n - c + 2) - 1)
    assert st["epochs"] == 2 * (n - c) + 1


# ----------------------------------------------------------------- N-Queens

def nq_brute(n):
    """Solutions and consistent-prefix count by enumerating permutations."""
    sols = 0
    for p in itertools.permutations(range(n)):
        if len({p[i] + i for i in range(n)}) == n and len({p[i] - i for i in range(n)}) == n:
            sols += 1
    nodes = 0
    for r in range(n + 1):
        for p in itertools.permutations(range(n), r):
            if len({p[i] + i for i in range(r)}) == r and len({p[i] - i for i in range(r)}) == r:
                nodes += 1
    return sols, nodes


def test_nqueens_known_counts():
    for n, sols in load_rows("nqueens_solutions.txt"):
        if n <= 11:
            assert oracle.nqueens(n)[0] == sols


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_nqueens_brute_force(n):
    sols, nodes = nq_brute(n)
    v, row_tasks, _ = oracle.nqueens(n)
    assert v == sols
    assert row_tasks == nodes


def test_nqueens_eight_brute_solutions():
    sols = sum(1 for p in itertools.permutations(range(8))
               if len({p[i] + i for i in range(8)}) == 8 and len({p[i] - i for i in range(8)}) == 8)
    assert sols == oracle.nqueens(8)[0] == 92
    assert oracle.nqueens(8)[1] == 2057     # the classic size of the 8-queens backtracking tree


@pytest.mark.parametrize("n", list(range(1, 12)))
def test_nqueens_tvm(n):
    sols, rows, joins = oracle.nqueens(n)
    r = oracle.tvm_run(oracle.NQUEENS, nq_n=n)
    st = r["stats"]
    assert st["root_result"] == sols
    assert st["tasks"] == rows + joins
    assert st["joins"] == joins
    if n >= 4:
        assert st["epochs"] == 2 * n + 1   # n+1 row levels, n join levels


# ----------------------------------------------------------------- mergesort

def leaf_count(n, leaf):
    if n <= leaf:
        return 1
    m = n // 2
    return leaf_count(m, leaf) + leaf_count(n - m, leaf)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 1023, 1024, 1025, 3000, 4096, 12345, 1 << 15])
def test_mergesort_matches_numpy(n):
    k = gen.keys_u32(7 + n, n)
    assert np.array_equal(oracle.mergesort(k), np.sort(k))
    r = oracle.tvm_run(oracle.MERGESORT, keys=k)
    assert np.array_equal(r["keys"], np.sort(k))
    leaves = leaf_count(n, 1024)
    st = r["stats"]
    assert st["tasks"] == 2 * leaves - 1 + (leaves - 1)
    assert st["maps"] == (leaves if n > 0 else 0) + (leaves - 1)


def test_mergesort_duplicates():
    rng = np.random.default_rng(3)
    k = rng.integers(0, 5, size=5000).astype(np.uint32)
    assert np.array_equal(oracle.mergesort(k, leaf=7), np.sort(k))
    assert np.array_equal(oracle.tvm_run(oracle.MERGESORT, keys=k, leaf=7)["keys"], np.sort(k))


@pytest.mark.parametrize("leaf", [1, 2, 3])
def test_mergesort_brute_force_small(leaf):
    for n in range(0, 7):
        for vals in itertools.product(range(3), repeat=n) if n <= 5 else [tuple(range(n))[::-1]]:
            k = np.array(vals, dtype=np.uint32)
            want = np.array(sorted(vals), dtype=np.uint32)
            assert np.array_equal(oracle.mergesort(k, leaf=leaf), want)
            assert np.array_equal(oracle.tvm_run(oracle.MERGESORT, keys=k, leaf=leaf)["keys"], want)


@pytest.mark.parametrize("log_leaves", [0, 1, 4, 6])
def test_mergesort_epochs_power_of_two(log_leaves):
    n = 1024 << log_leaves
    st = oracle.tvm_run(oracle.MERGESORT, keys=gen.keys_u32(1, n))["stats"]
    assert st["epochs"] == 2 * log_leaves + 1
    assert st["tasks"] == (2 << log_leaves) - 1 + (1 << log_leaves) - 1


# ----------------------------------------------------------------- BFS

def random_graph(nv, p, seed):
    rng = np.random.default_rng(seed)
    a = rng.random((nv, nv)) < p
    a = np.triu(a, 1)
    a = a | a.T
    row_ptr = np.zeros(nv + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum(a.sum(1))
    col = np.concatenate([np.nonzero(a[i])[0] for i in range(nv)] + [np.zeros(0, int)]).astype(np.int32)
    return a, row_ptr, col


def floyd_warshall_hops(a):
    nv = a.shape[0]
    inf = 10 ** 9
    d = np.where(a, 1, inf).astype(np.int64)
    np.fill_diagonal(d, 0)
    for k in range(nv):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    return np.where(d >= inf, -1, d)


@pytest.mark.parametrize("nv,p,seed", [(1, 0.0, 0), (5, 0.0, 1), (12, 0.2, 2), (40, 0.05, 3),
                                       (64, 0.03, 4), (64, 0.3, 5)])
def test_bfs_floyd_warshall(nv, p, seed):
    a, row_ptr, col = random_graph(nv, p, seed)
    d = floyd_warshall_hops(a)
    for src in {0, nv - 1}:
        level, reached = oracle.bfs(row_ptr, col, src)
        assert np.array_equal(level, d[src])
        assert reached == int((d[src] >= 0).sum())
        r = oracle.tvm_run(oracle.BFS, row_ptr=row_ptr, col=col, src=src)
        assert np.array_equal(r["level"], d[src])
        st = r["stats"]
        assert st["tasks"] == reached
        assert st["epochs"] == int(d[src].max()) + 1
        # epoch k runs exactly the vertices at distance k
        for t in r["trace"]:
            assert t["valid"] == int((d[src] == t["cen"]).sum())


def test_bfs_rmat_scipy():
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    row_ptr, col, info = gen.rmat(10, 16, seed=2)
    nv = info["nv"]
    m = csr_matrix((np.ones(col.shape[0]), col, row_ptr), shape=(nv, nv))
    d = shortest_path(m, unweighted=True, indices=[0])[0]
    want = np.where(np.isinf(d), -1, d).astype(np.int32)
    level, reached = oracle.bfs(row_ptr, col, 0)
    assert np.array_equal(level, want)
    r = oracle.tvm_run(oracle.BFS, row_ptr=row_ptr, col=col, src=0)
    assert np.array_equal(r["level"], want)
    assert r["stats"]["tasks"] == reached
    assert r["stats"]["epochs"] == int(want.max()) + 1


# ----------------------------------------------------------------- Fig. 3 worked example

@pytest.mark.parametrize("null_under", ["B", "C"])
def test_fig3_postorder_trace(null_under):
    # A=0 with children B=1, C=2; three leaves D, E, F below B and C with one NULL slot.
    if null_under == "B":
        left = np.array([1, 3, 4, -1, -1, -1]); right = np.array([2, -1, 5, -1, -1, -1])
    else:
        left = np.array([1, 3, 5, -1, -1, -1]); right = np.array([2, 4, -1, -1, -1, -1])
    r = oracle.tvm_run(oracle.POSTORDER, left=left, right=right)
    rows = load_rows("fig3_postorder_trace.txt")
    tr = r["trace"]
    assert len(tr) == len(rows)
    assert r["stats"]["final_slots"] == 0
    for (e, cen, lo, hi, valid, forks, joined), t in zip(rows, tr):
        assert (t["cen"], t["lo"], t["hi"], t["valid"], t["forks"], t["joined"]) == \
            (cen, lo, hi, valid, forks, joined), e
    # postorder: every node is visited after its children
    ve = r["visit_epoch"]
    for v in range(6):
        for c in (left[v], right[v]):
            if c >= 0:
                assert ve[v] > ve[c]


def test_traversal_orders_random_tree():
    left, right = gen.binary_tree(11, 300)
    post = oracle.tvm_run(oracle.POSTORDER, left=left, right=right)["visit_epoch"]
    pre = oracle.tvm_run(oracle.PREORDER, left=left, right=right)["visit_epoch"]
    depth = np.full(300, -1)
    depth[0] = 0
    stack = [0]
    while stack:
        v = stack.pop()
        for c in (left[v], right[v]):
            if c >= 0:
                depth[c] = depth[v] + 1
                stack.append(c)
    assert (depth >= 0).all()
    assert np.array_equal(pre, depth)                 # preorder visits at its forward epoch
    for v in range(300):
        for c in (left[v], right[v]):
            if c >= 0:
                assert post[v] > post[c]


# ----------------------------------------------------------------- SSSP (Sec. 6.3)

def floyd_warshall_weighted(nv, row_ptr, col, weight):
    """All-pairs shortest path lengths by Floyd-Warshall (brute force, int64,
    -1 = unreachable); the minimum weight is kept for parallel edges."""
    inf = np.int64(1) << 60  # inf + inf stays inside int64
    d = np.full((nv, nv), inf, dtype=np.int64)
    for v in range(nv):
        for e in range(row_ptr[v], row_ptr[v + 1]):
            d[v, col[e]] = min(d[v, col[e]], int(weight[e]))
    np.fill_diagonal(d, 0)
    for k in range(nv):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    return d, inf


def weighted_random_graph(nv, p, seed, wmax, directed):
    """Erdos-Renyi graph in CSR with weights in [0, wmax] (zero weights included)."""
    rng = np.random.default_rng(seed)
    a = rng.random((nv, nv)) < p
    np.fill_diagonal(a, False)
    if not directed:
        a = np.triu(a, 1)
        a = a | a.T
    wm = rng.integers(0, wmax + 1, size=(nv, nv)).astype(np.uint32)
    if not directed:
        wm = np.triu(wm, 1)
        wm = wm + wm.T
    row_ptr = np.zeros(nv + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum(a.sum(1))
    cols = [np.nonzero(a[i])[0] for i in range(nv)]
    col = np.concatenate(cols + [np.zeros(0, int)]).astype(np.int32)
    weight = np.concatenate([wm[i, cols[i]] for i in range(nv)] + [np.zeros(0, np.uint32)]).astype(np.uint32)
    return row_ptr, col, weight


def check_sssp_invariants(row_ptr, col, weight, src, dist):
    """dist[src] = 0; no edge can shorten a distance; every other reached vertex
    has an incoming edge that attains its distance (the shortest-path tree)."""
    nv = row_ptr.shape[0] - 1
    inf = oracle.SSSP_INF
    assert dist[src] == 0
    src_of = np.repeat(np.arange(nv), np.diff(row_ptr))
    ds, du = dist[src_of], dist[col]
    ok = ds != inf
    cand = ds[ok] + weight[ok].astype(np.uint64)
    assert (du[ok] <= cand).all()
    tight = np.zeros(nv, dtype=bool)
    tight[col[ok][du[ok] == cand]] = True
    reached = dist != inf
    reached[src] = False
    assert tight[reached].all()


@pytest.mark.parametrize("nv,p,seed,wmax,directed", [(1, 0.0, 0, 5, False), (6, 0.0, 1, 5, True),
                                                     (12, 0.25, 2, 9, True), (40, 0.08, 3, 100, False),
                                                     (64, 0.05, 4, 1, True), (64, 0.2, 5, 1000, False)])
def test_sssp_floyd_warshall(nv, p, seed, wmax, directed):
    row_ptr, col, weight = weighted_random_graph(nv, p, seed, wmax, directed)
    d, inf = floyd_warshall_weighted(nv, row_ptr, col, weight)
    for src in {0, nv - 1}:
        want = d[src].astype(np.uint64)
        want[d[src] >= inf] = oracle.SSSP_INF
        dist, reached = oracle.sssp_dijkstra(row_ptr, col, weight, src)
        assert np.array_equal(dist, want)
        assert reached == int((d[src] < inf).sum())
        wl, rounds, relaxed = oracle.sssp_worklist(row_ptr, col, weight, src)
        assert np.array_equal(wl, want)
        assert relaxed >= reached and rounds >= 1
        check_sssp_invariants(row_ptr, col, weight, src, dist)


def test_sssp_rmat_scipy_and_worklist():
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra
    row_ptr, col, info = gen.rmat(10, 16, seed=2)
    nv = info["nv"]
    weight = gen.weights(3, row_ptr, col)
    assert weight.min() >= 1 and weight.max() <= 255
    m = csr_matrix((weight.astype(np.float64), col, row_ptr), shape=(nv, nv))
    d = dijkstra(m, indices=[0])[0]
    want = np.where(np.isinf(d), 0, d).astype(np.uint64)
    want[np.isinf(d)] = oracle.SSSP_INF
    dist, reached = oracle.sssp_dijkstra(row_ptr, col, weight, 0)
    assert np.array_equal(dist, want)
    wl, rounds, relaxed = oracle.sssp_worklist(row_ptr, col, weight, 0)
    assert np.array_equal(wl, want)
    assert rounds > int(oracle.bfs(row_ptr, col, 0)[0].max())   # weights make paths longer than hops
    check_sssp_invariants(row_ptr, col, weight, 0, dist)


def test_sssp_unit_weights_are_bfs_levels():
    row_ptr, col, info = gen.rmat(11, 8, seed=7)
    level, _ = oracle.bfs(row_ptr, col, 3)
    dist, _ = oracle.sssp_dijkstra(row_ptr, col, np.ones(col.shape[0], np.uint32), 3)
    want = np.maximum(level, 0).astype(np.uint64)
    want[level < 0] = oracle.SSSP_INF
    assert np.array_equal(dist, want)
    wl, rounds, relaxed = oracle.sssp_worklist(row_ptr, col, np.ones(col.shape[0], np.uint32), 3)
    assert np.array_equal(wl, want)
    assert rounds == int(level.max()) + 1 and relaxed == int((level >= 0).sum())  # BFS levels, each once


def test_sssp_source_out_of_range_and_isolated():
    row_ptr = np.array([0, 1, 2, 2], np.int32)
    col = np.array([1, 0], np.int32)
    w = np.array([4, 4], np.uint32)
    dist, reached = oracle.sssp_dijkstra(row_ptr, col, w, 5)
    assert reached == 0 and (dist == oracle.SSSP_INF).all()
    dist, reached = oracle.sssp_dijkstra(row_ptr, col, w, 2)
    assert reached == 1 and dist[2] == 0 and dist[0] == dist[1] == oracle.SSSP_INF


# ------------------------------------------------------------ FFT (Sec. 6.2, Fig. 6)

def fft_input(seed, n):
    return gen.signal(seed, n).astype(np.complex128)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 64])
def test_dft_closed_forms(n):
    j = np.arange(n)
    # a constant sums to n at frequency 0 and cancels elsewhere
    X = oracle.dft(np.full(n, 2.0 - 1.0j))
    want = np.zeros(n, complex)
    want[0] = n * (2.0 - 1.0j)
    assert np.allclose(X, want, atol=1e-12 * n)
    # the tone exp(+2 pi i f j / n) lands on bin f alone (a sign error would put it on n - f)
    for f in range(n):
        X = oracle.dft(np.exp(2j * np.pi * f * j / n))
        want = np.zeros(n, complex)
        want[f] = n
        assert np.allclose(X, want, atol=1e-10 * n)
    # a geometric sequence r^j has the closed form (1 - r^n) / (1 - r exp(-2 pi i k / n))
    r = 0.9 * np.exp(0.3j)
    X = oracle.dft(r ** j)
    k = np.arange(n)
    assert np.allclose(X, (1 - r ** n) / (1 - r * np.exp(-2j * np.pi * k / n)), atol=1e-11 * n)


@pytest.mark.parametrize("n", [1, 7, 64, 1000])
def test_dft_matches_numpy_and_theorems(n):
    x = fft_input(11, n)
    X = oracle.dft(x)
    scale = np.linalg.norm(X) + 1.0
    assert np.linalg.norm(X - np.fft.fft(x)) <= 1e-12 * n * scale
    # Parseval: sum |x|^2 = sum |X|^2 / n
    assert abs(np.sum(abs(x) ** 2) - np.sum(abs(X) ** 2) / n) <= 1e-10 * np.sum(abs(x) ** 2) + 1e-300
    # shift theorem: x[j - m] <-> X[k] exp(-2 pi i k m / n)
    m = n // 3
    Xs = oracle.dft(np.roll(x, m))
    assert np.linalg.norm(Xs - X * np.exp(-2j * np.pi * np.arange(n) * m / n)) <= 1e-11 * n * scale
    # linearity
    y = fft_input(12, n)
    assert np.linalg.norm(oracle.dft(x + 2 * y) - (X + 2 * oracle.dft(y))) <= 1e-11 * n * scale
    # single outputs equal the full transform's
    ks = [0, n - 1, n // 2]
    assert np.array_equal(oracle.dft_at(x, ks), X[ks])


def fft_tvm_counts(n, leaf, cutoff):
    """The FFT task tree in closed form: depth D = log2(n / leaf) levels of
    forks (2^d tasks at depth d), 2^D leaves, one combine per internal task."""
    D = max(0, n.bit_length() - 1 - (leaf.bit_length() - 1)) if n > leaf else 0
    maps = sum(2 ** d for d in range(D) if (n >> d) > cutoff)
    return {"epochs": 2 * D + 1, "tasks": 2 ** (D + 1) - 1 + 2 ** D - 1, "forks": 2 ** (D + 1) - 2,
            "joins": 2 ** D - 1, "maps": maps, "peak_slots": 2 ** (D + 1) - 1, "final_slots": 0}, D


@pytest.mark.parametrize("lg", [0, 1, 2, 3, 5, 8, 10])
@pytest.mark.parametrize("leaf,cutoff", [(1, 0), (2, 4), (4, 1 << 20), (16, 32)])
def test_fft_tvm_matches_dft_and_closed_forms(lg, leaf, cutoff):
    n = 1 << lg
    x = fft_input(lg * 7 + leaf, n)
    r = oracle.tvm_run(oracle.FFT, x=x, fft_leaf=leaf, fft_cutoff=cutoff)
    want = np.fft.fft(x)
    assert np.linalg.norm(r["X"] - want) <= 1e-14 * (lg + 1) * np.linalg.norm(want)
    counts, D = fft_tvm_counts(n, leaf, cutoff)
    for key, v in counts.items():
        assert r["stats"][key] == v, key
    # the epochs: fork levels 0..D, then the join ranges revisited bottom-up
    tr = r["trace"]
    for i, t in enumerate(tr):
        d = i if i <= D else 2 * D - i
        assert (t["cen"], t["lo"], t["hi"], t["valid"]) == (d, 2 ** d - 1, 2 ** (d + 1) - 1, 2 ** d)
        assert t["forks"] == (2 ** (d + 1) if i < D else 0)
        assert t["joined"] == (1 if i < D else 0)
        assert t["maps"] == (2 ** d if i > D and (n >> d) > cutoff else 0)


def test_fft_tvm_single_leaf_is_the_definition():
    x = fft_input(5, 16)
    r = oracle.tvm_run(oracle.FFT, x=x, fft_leaf=16)
    assert r["stats"]["tasks"] == 1 and r["stats"]["epochs"] == 1
    assert np.allclose(r["X"], oracle.dft(x), rtol=0, atol=1e-13)


# ------------------------------------------------------------ the user-program example (chunked sum)

@pytest.mark.parametrize("chunk,arity,k", [(4096, 8, 0), (4096, 8, 1), (4096, 8, 3), (1000, 2, 5), (7, 3, 4)])
def test_chunk_sum_tree_perfect_closed_forms(chunk, arity, k):
    """n = chunk * arity^k: a perfect arity-ary tree of depth k."""
    st, tr = oracle.chunk_sum_tree(chunk * arity ** k, chunk, arity)
    internal = (arity ** k - 1) // (arity - 1)
    assert st["maps"] == arity ** k and st["joins"] == internal
    assert st["epochs"] == 2 * k + 1 and st["tasks"] == arity ** k + 2 * internal
    assert st["peak_slots"] == arity ** k + internal
    assert [t["valid"] for t in tr[:k + 1]] == [arity ** d for d in range(k + 1)]


def test_chunk_sum_tree_brute_force_leaves():
    """The leaves partition [0, n) into ranges of at most chunk keys, every
    internal range has the stated arity, for many small (n, chunk, arity)."""
    for n in range(0, 60):
        for chunk in (1, 2, 5, 16):
            for arity in (2, 3, 8):
                st, tr = oracle.chunk_sum_tree(n, chunk, arity)
                # enumerate by hand: a plain recursion of the definition
                leaves, internal, depth = [], 0, 0

                def rec(lo, hi, d):
                    nonlocal internal, depth
                    depth = max(depth, d)
                    if hi - lo <= chunk:
                        leaves.append((lo, hi))
                        return
                    internal += 1
                    kk = min(arity, -(-(hi - lo) // chunk))
                    cuts = [lo + (hi - lo) * i // kk for i in range(kk + 1)]
                    for a, b in zip(cuts, cuts[1:]):
                        rec(a, b, d + 1)

                rec(0, n, 0)
                assert sorted(leaves) == leaves and leaves[0][0] == 0 and leaves[-1][1] == n
                assert all(b - a <= chunk for a, b in leaves) and all(a < b for a, b in leaves[1:] if n)
                assert st["maps"] == sum(1 for a, b in leaves if b > a) and st["joins"] == internal
                assert st["epochs"] == 2 * depth + 1
