"""The CPU context baseline (the paper's method on the host) computes the
oracle's products."""
import numpy as np
import pytest

import oracle
from paper_0901_1413_gb300 import context_cpu, inputs

FIELDS = (2, 3, 4, 5, 7)


@pytest.mark.parametrize("q", FIELDS)
@pytest.mark.parametrize("mln,k", [((1, 1, 1), 3), ((37, 100, 70), 4), ((64, 65, 129), 8), ((200, 333, 150), 7),
                                   ((5, 0, 9), 2)])
def test_matches_oracle(q, mln, k):
    m, l, n = mln
    A = inputs.uniform(q, m, l, seed=m + q, stream=inputs.STREAM_A)
    B = inputs.uniform(q, l, n, seed=m + q, stream=inputs.STREAM_B)
    C, ms = context_cpu.matmul(q, A, B, k=k, threads=2)
    assert np.array_equal(C, oracle.matmul(q, A, B))
    assert ms >= 0


@pytest.mark.parametrize("q", (3, 5))
def test_threads_and_default_k(q):
    A = inputs.uniform(q, 300, 260, seed=7, stream=inputs.STREAM_A)
    B = inputs.uniform(q, 260, 190, seed=7, stream=inputs.STREAM_B)
    want = oracle.matmul(q, A, B)
    for threads in (1, 3):
        assert np.array_equal(context_cpu.matmul(q, A, B, threads=threads)[0], want)
    assert 2 <= context_cpu.default_k(q, 2500) <= 10


def test_rejects_bad_input():
    with pytest.raises(ValueError):
        context_cpu.matmul(6, np.zeros((2, 2), np.uint8), np.zeros((2, 2), np.uint8))
    with pytest.raises(ValueError):
        context_cpu.matmul(3, np.full((2, 2), 3, np.uint8), np.zeros((2, 2), np.uint8))
