"""Plants plausible mistakes into a copy of the oracle and checks that the
pins of test_oracle.py catch every one (CPU only).  The planted copies are
built in a temporary directory; the real oracle is restored afterwards."""
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle
import test_oracle as pins

MUTANTS = {
    # a join drops one child's result
    "fib_sum_drops_term": ("m->result[m->link[s]] + m->result[m->link[s] + 1]", "m->result[m->link[s]]"),
    # Phase 3 pushes the fork range below the join range (wrong LIFO order)
    "phase3_order_swapped": (
        "        if (m.join_scheduled) push(&m, r.cen, r.lo, r.hi);\n"
        "        if (forked) push(&m, r.cen + 1, (uint32_t)old_next, (uint32_t)m.next);\n",
        "        if (forked) push(&m, r.cen + 1, (uint32_t)old_next, (uint32_t)m.next);\n"
        "        if (m.join_scheduled) push(&m, r.cen, r.lo, r.hi);\n"),
    # forked children are tagged for the wrong epoch
    "fork_epoch_off_by_one": ("m->code[s] = (m->cen + 1) * NUM_TASK_TYPES + type;",
                              "m->code[s] = (m->cen + 2) * NUM_TASK_TYPES + type;"),
    # the nextFreeCore decrease of Sec. 5.3 is lost
    "no_reclaim": ("            m.next = r.lo;\n", "\n"),
    # a diagonal shifts the wrong way
    "nq_diagonal_sign": ("nd1 = ((d1 | b) << 1) & mask", "nd1 = ((d1 | b) >> 1) & mask"),
    # the merge forgets the right half's tail
    "merge_drops_tail": ("        while (j < op->c) m->tmp[o++] = k[j++];\n", "\n"),
    # BFS labels a claimed vertex with the wrong level
    "bfs_level_off_by_one": ("p->level[u] = (int32_t)(m->cen + 1);", "p->level[u] = (int32_t)(m->cen + 2);"),
    # the footnote-2 range test excludes the last task type
    "encoding_upper_bound": ("if (c < lo_code || c > hi_code) continue;", "if (c < lo_code || c >= hi_code) continue;"),
    # a join reads the wrong sibling
    "nq_sum_wrong_index": ("sum += m->result[m->link[s] + i];", "sum += m->result[m->link[s] + i + 1];"),
    # Dijkstra's heap keeps the wrong end on top
    "sssp_heap_order": ("        if (h[p].d <= x.d) break;", "        if (h[p].d >= x.d) break;"),
    # a relaxation adds one to every path
    "sssp_relax_plus_one": ("const uint64_t nd = it.d + weight[e];", "const uint64_t nd = it.d + weight[e] + 1u;"),
    # the worklist never revisits a vertex whose distance dropped again
    "sssp_worklist_no_requeue": ("if (queued[u] != r) { queued[u] = r; out[nout++] = u; }",
                                 "if (queued[u] < 0) { queued[u] = r; out[nout++] = u; }"),
    # the plain recursion counts calls wrongly
    "fib_calls_skip": ("    (*calls)++;\n    if (n < 2) return n;", "    if (n < 2) return n;\n    (*calls)++;"),
    # the definition's kernel has the wrong sign
    "dft_kernel_sign": ("const double ang = -2.0 * M_PI * (double)((j * k) % n) / (double)n;\n    const double c",
                        "const double ang = 2.0 * M_PI * (double)((j * k) % n) / (double)n;\n    const double c"),
    # the definition pairs j with k by a sum instead of a product
    "dft_index_sum": ("(double)((j * k) % n) / (double)n;\n    const double c",
                      "(double)((j + k) % n) / (double)n;\n    const double c"),
    # the combine's twiddle turns the wrong way
    "fft_twiddle_sign": ("const double ang = -2.0 * M_PI * (double)k / (double)n, wr",
                         "const double ang = 2.0 * M_PI * (double)k / (double)n, wr"),
    # the second half of a combine adds instead of subtracting
    "fft_combine_second_half": ("        od[0] = er - tr;\n", "        od[0] = er + tr;\n"),
    # output blocks are placed with the bit weights reversed
    "fft_block_bit_order": ("if ((o >> b) & 1u) pos += N >> (b + 1);", "if ((o >> b) & 1u) pos += N >> (d - b);"),
    # a leaf drops the imaginary part of its input
    "fft_leaf_drops_imag": (" - p->fft_x[2 * src + 1] * sin(ang);", ";"),
}


def run_pins():
    """The pins, called directly; any AssertionError/RuntimeError means caught."""
    for n in (5, 12, 20):
        pins.test_fib_value_and_calls(n)
        pins.test_fib_tvm_closed_forms(n)
    pins.test_fib_cutoff_closed_forms(20, 12)
    pins.test_nqueens_known_counts()
    for n in range(1, 8):
        pins.test_nqueens_brute_force(n)
        pins.test_nqueens_tvm(n)
    pins.test_mergesort_matches_numpy(3000)
    pins.test_mergesort_brute_force_small(2)
    pins.test_bfs_floyd_warshall(40, 0.05, 3)
    pins.test_sssp_floyd_warshall(40, 0.08, 3, 100, False)
    pins.test_sssp_rmat_scipy_and_worklist()
    pins.test_fig3_postorder_trace("B")
    pins.test_traversal_orders_random_tree()
    for n in (1, 8, 12):
        pins.test_dft_closed_forms(n)
    pins.test_dft_matches_numpy_and_theorems(64)
    for lg in (1, 3, 8):
        pins.test_fft_tvm_matches_dft_and_closed_forms(lg, 2, 4)
        pins.test_fft_tvm_matches_dft_and_closed_forms(lg, 1, 0)
        pins.test_fft_tvm_matches_dft_and_closed_forms(lg, 16, 32)


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


def test_unmutated_oracle_passes_pins():
    run_pins()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, workdir):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = os.path.join(str(workdir), f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = path[:-2] + ".so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", path, "-o", so, "-lm"])
    saved = oracle._load()
    oracle._lib = oracle._bind(ctypes.CDLL(so))
    try:
        with pytest.raises((AssertionError, RuntimeError)):
            run_pins()
    finally:
        oracle._lib = saved
