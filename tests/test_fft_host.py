"""Host-side sizing of the FFT program (CPU only: no kernel runs).

trees_job_slots must give the peak task-vector need of the FFT task tree,
2^(D+1) - 1 slots for D = log2(n / leaf), which the oracle's TVM run
measures independently."""
import numpy as np
import pytest

import oracle
import paper_1608_00571_b300 as T


def fft_job(n, leaf):
    return T.make_job(T.TREES_PROG_FFT, n=n, leaf=leaf, fft_in=8, fft_out=16 * n + 8)


@pytest.mark.parametrize("leaf", [0, 1, 2, 4, 8, 16])
def test_fft_job_slots_match_the_oracle_tree(leaf):
    for lg in range(0, 11):
        n = 1 << lg
        slots, exact = T.trees_job_slots(fft_job(n, leaf))
        sim = oracle.tvm_run(oracle.FFT, x=np.zeros(n), fft_leaf=leaf or 16)
        assert exact and slots == sim["stats"]["peak_slots"], (n, leaf)


def test_fft_job_slots_closed_form_up_to_the_maximum():
    for lg in range(0, 26):
        for leaf in (1, 16):
            d = max(0, lg - int(np.log2(leaf)))
            assert T.trees_job_slots(fft_job(1 << lg, leaf))[0] == 2 ** (d + 1) - 1
