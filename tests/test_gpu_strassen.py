"""Strassen-Winograd levels over the base-field kernels: bit-identical to the
direct product, and exact against the oracle on sampled rows."""
import numpy as np
import pytest
import torch

import oracle
from oracle import encoding
from paper_0901_1413_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = (2, 3, 4, 5, 7)


def operands(fq, q, m, l, n, seed):
    A = inputs.uniform_torch(q, m, l, seed=seed, stream=inputs.STREAM_A)
    B = inputs.uniform_torch(q, l, n, seed=seed, stream=inputs.STREAM_B)
    return A, B, fq.pack(q, A), fq.pack(q, B)


def check(fq, q, m, l, n, levels, seed=0, rows=8, **kw):
    A, B, a, b = operands(fq, q, m, l, n, seed)
    assert fq.strassen_levels(q, m, l, n, strassen=levels, path=kw.get("path", 0)) == levels
    c1 = fq.matmul(a, b, strassen=levels, **kw)
    c0 = fq.matmul(a, b, strassen=-1, **kw)
    assert fq.status() == fq.OK
    assert torch.equal(c1.data, c0.data)          # canonical planes, bit for bit
    C = fq.unpack(c1).cpu().numpy()
    sample = np.random.default_rng(seed + q).choice(m, size=rows, replace=False)
    Ah = A[torch.from_numpy(sample).cuda()].cpu().numpy()
    assert np.array_equal(C[sample], oracle.matmul(q, Ah, B.cpu().numpy()))
    return c1


@pytest.mark.parametrize("q", FIELDS)
def test_one_level_square(fq, q):
    check(fq, q, 2048, 2048, 2048, 1, seed=q)


@pytest.mark.parametrize("q", (3, 5))
def test_one_level_rectangular(fq, q):
    check(fq, q, 4096, 2048, 6144, 1, seed=10 + q)


def test_two_levels(fq):
    check(fq, 3, 4096, 4096, 4096, 2, seed=20)


def test_full_oracle_through_one_level(fq):
    """Every entry of a 2048^3 F_7 product by one level against the oracle."""
    A, B, a, b = operands(fq, 7, 2048, 2048, 2048, seed=31)
    c = fq.matmul(a, b, strassen=1)
    got = fq.unpack(c).cpu().numpy()
    assert np.array_equal(got, oracle.matmul(7, A.cpu().numpy(), B.cpu().numpy()))
    words = c.planes_view().cpu().numpy().view(np.uint64)
    assert np.array_equal(words, encoding.pack(7, got))    # canonical codes


@pytest.mark.parametrize("q", (3, 5))
def test_tensor_core_base_products(fq, q):
    check(fq, q, 2048, 2048, 2048, 1, seed=40 + q, path=fq.PATH_MMA)


def test_extension_field_base_products(fq):
    """F_9's three F_3 products each take a level."""
    A, B, a, b = operands(fq, 9, 2048, 2048, 2048, seed=50)
    c1 = fq.matmul(a, b, strassen=1)
    c0 = fq.matmul(a, b, strassen=-1)
    assert torch.equal(c1.data, c0.data)
    rows = [0, 777, 2047]
    got = fq.unpack(c1).cpu().numpy()[rows]
    assert np.array_equal(got, oracle.matmul(9, A[rows].cpu().numpy(), B.cpu().numpy()))


def test_shapes_that_do_not_split(fq):
    """A requested level is skipped where a half would not be whole pitches."""
    assert fq.strassen_levels(3, 3000, 2048, 2048, strassen=1) == 0
    assert fq.strassen_levels(3, 2048, 2048, 1024, strassen=1) == 0
    assert fq.strassen_levels(3, 4096, 4096, 2048, strassen=3) == 1
    A, B, a, b = operands(fq, 3, 3000, 2048, 2048, seed=60)
    got = fq.unpack(fq.matmul(a, b, strassen=1)).cpu().numpy()
    rows = [0, 2999]
    assert np.array_equal(got[rows], oracle.matmul(3, A[rows].cpu().numpy(), B.cpu().numpy()))


def test_time_model_levels(fq):
    """On GB300 the model takes one level for F_3 M4RM products at 16384 and
    none at 8192; the tcgen05 products stay direct."""
    M = fq.PATH_M4RM
    assert fq.strassen_levels(3, 8192, 8192, 8192, path=M) == 0
    assert fq.strassen_levels(3, 16384, 16384, 16384, path=M) >= 1
    assert fq.strassen_levels(3, 16384, 16384, 16384, path=M, strassen=-1) == 0
    assert fq.strassen_levels(3, 16384, 16384, 16384, path=fq.PATH_MMA) == 0
    assert fq.strassen_levels(9, 16384, 16384, 16384) == 0    # extension fields: per base product


def test_graph_capture(fq):
    A, B, a, b = operands(fq, 3, 2048, 2048, 2048, seed=70)
    c = fq.empty(3, 2048, 2048)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        fq.matmul(a, b, out=c, strassen=1, stream=stream)
    torch.cuda.synchronize()
    want = c.data.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fq.matmul(a, b, out=c, strassen=1, stream=stream)
    c.data.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(c.data, want)
    assert fq.status() == fq.OK


def test_release_scratch(fq):
    A, B, a, b = operands(fq, 3, 2048, 2048, 2048, seed=75)
    c0 = fq.matmul(a, b, strassen=1)
    assert fq.load().fq_release_scratch() == fq.OK
    c1 = fq.matmul(a, b, strassen=1)                 # the pool grows again
    assert torch.equal(c0.data, c1.data)
    assert fq.status() == fq.OK


@pytest.mark.slow
def test_f3_16384_auto_level_matches_direct(fq):
    A, B, a, b = operands(fq, 3, 16384, 16384, 16384, seed=80)
    assert fq.strassen_levels(3, 16384, 16384, 16384, k=8) >= 1
    c1 = fq.matmul(a, b, k=8)
    c0 = fq.matmul(a, b, path=fq.PATH_MMA, strassen=-1)     # the tcgen05 form
    assert torch.equal(c1.data, c0.data)
