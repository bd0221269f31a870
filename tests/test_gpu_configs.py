"""The benchmark workloads at full size, on both forced paths.

For every workload the Four-Russians path (Section 2, FQ_PATH_M4RM) and the
exact tensor-core contraction (FQ_PATH_MMA) must give identical planes, and the
product must equal the oracle on 256 sampled rows and 256 sampled columns
(the last row and column among them, so ragged tile edges are covered) and
pass a 32-trial Freivalds check, which a wrong product passes with probability
at most q^-32.  C = AB is unique, so any difference is an error.

Workloads: F_3 n = 4096, 8192, 16384 and n = 8192 with A 90% zeros; F_5, F_7
and GF(4) at n = 8192; F_5 32768^3; F_3 65536 x 4096 x 4096.  At 4096^3 every
field is also compared with the full oracle product on both paths.

Integer work: every comparison is bit-exact (zero tolerance)."""
import numpy as np
import pytest
import torch

import oracle
from paper_0901_1413_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SAMPLES = 256
TRIALS = 32

WORKLOADS = [
    (3, 4096, 4096, 4096, "uniform"),
    (3, 8192, 8192, 8192, "uniform"),
    (3, 16384, 16384, 16384, "uniform"),
    (3, 8192, 8192, 8192, "sparse90"),
    (5, 8192, 8192, 8192, "uniform"),
    (7, 8192, 8192, 8192, "uniform"),
    (4, 8192, 8192, 8192, "uniform"),
    (5, 32768, 32768, 32768, "uniform"),
    (3, 65536, 4096, 4096, "uniform"),
]


def _draw(q, m, l, n, law, seed):
    """A and B drawn on the device (the bench's generator), with one sampled
    row of each redrawn on the host to show the two agree."""
    gen = inputs.sparse_torch if law == "sparse90" else inputs.uniform_torch
    A = gen(q, m, l, seed=seed, stream=inputs.STREAM_A, device="cuda")
    B = inputs.uniform_torch(q, l, n, seed=seed, stream=inputs.STREAM_B, device="cuda")
    host = inputs.sparse if law == "sparse90" else inputs.uniform
    assert np.array_equal(host(q, 1, l, seed=seed, stream=inputs.STREAM_A, row0=m - 1)[0], A[m - 1].cpu().numpy())
    assert np.array_equal(inputs.uniform(q, 1, n, seed=seed, stream=inputs.STREAM_B, row0=l // 2)[0],
                          B[l // 2].cpu().numpy())
    return A, B


def _sample(rng, size):
    idx = rng.choice(size, size=min(SAMPLES, size), replace=False)
    idx[0] = size - 1
    return np.unique(idx)


@pytest.mark.parametrize("q,m,l,n,law", WORKLOADS, ids=lambda v: str(v))
def test_workload_both_paths_sampled_oracle_and_freivalds(fq, q, m, l, n, law):
    seed = 5
    A, B = _draw(q, m, l, n, law, seed)
    a, b = fq.pack(q, A), fq.pack(q, B)
    c_m4rm = fq.matmul(a, b, path=fq.PATH_M4RM)
    c_tc = fq.matmul(a, b, path=fq.PATH_MMA)
    assert fq.status() == fq.OK
    assert torch.equal(c_m4rm.data, c_tc.data), "the two paths differ"
    del c_tc, a, b
    C = fq.unpack(c_m4rm).cpu().numpy()
    del c_m4rm
    Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
    del A, B
    torch.cuda.empty_cache()
    rng = np.random.default_rng(m + 3 * n + q)
    rows, cols = _sample(rng, m), _sample(rng, n)
    assert np.array_equal(C[rows], oracle.matmul_rows(q, Ah, Bh, rows)), "sampled rows"
    assert np.array_equal(C[:, cols], oracle.matmul_cols(q, Ah, Bh, cols)), "sampled columns"
    assert oracle.freivalds(q, Ah, Bh, C, trials=TRIALS, seed=q + m), "Freivalds"


@pytest.mark.parametrize("q", (2, 3, 4, 5, 7))
def test_4096_full_oracle_both_paths(fq, q):
    """Every field at 4096^3: the whole product against the oracle, on the
    Four-Russians path and on the tensor-core path."""
    m = l = n = 4096
    A = inputs.uniform(q, m, l, seed=q, stream=inputs.STREAM_A)
    B = inputs.uniform(q, l, n, seed=q, stream=inputs.STREAM_B)
    a, b = fq.pack(q, torch.from_numpy(A).cuda()), fq.pack(q, torch.from_numpy(B).cuda())
    want = oracle.matmul(q, A, B)
    for path in (fq.PATH_M4RM, fq.PATH_MMA):
        got = fq.unpack(fq.matmul(a, b, path=path)).cpu().numpy()
        assert fq.status() == fq.OK
        assert np.array_equal(got, want), "path %d: first mismatch at %s" % (path, np.argwhere(got != want)[:3].tolist())
