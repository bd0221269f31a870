"""Extension fields F_{p^n} (Section 4.3's matrix-level products) and GF(4) by
three F_2 products: the CUDA path against the oracle through the C ABI,
bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from oracle import encoding
from oracle.fields import EXTENSIONS
from paper_0901_1413_gb300 import inputs
from tests import pins

pytestmark = pytest.mark.gpu

EXT = (8, 9, 25, 27, 49, 125)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def packed_words(x):
    v = x.planes_view().cpu().numpy().view(np.uint64)
    w = (x.cols + 63) // 64
    return v[:, :, :w], v[:, :, w:]


def check(fq, q, m, l, n, seed, sparse=False, **kw):
    A = (inputs.sparse if sparse else inputs.uniform)(q, m, l, seed=seed, stream=inputs.STREAM_A)
    B = inputs.uniform(q, l, n, seed=seed, stream=inputs.STREAM_B)
    c = fq.matmul(fq.pack(q, to_dev(A)), fq.pack(q, to_dev(B)), **kw)
    got = fq.unpack(c).cpu().numpy()
    assert fq.status() == fq.OK
    want = oracle.matmul(q, A, B)
    assert np.array_equal(got, want), "first mismatch at %s" % (np.argwhere(got != want)[:3].tolist(),)
    words, pad = packed_words(c)
    assert np.array_equal(words, encoding.pack(q, want))      # canonical coefficient codes
    assert not pad.any()
    return c


@pytest.mark.parametrize("q", EXT)
@pytest.mark.parametrize("shape", [(1, 1), (3, 65), (33, 1000), (2, 1100)])
def test_pack_is_coefficient_planes(fq, q, shape):
    R = inputs.uniform(q, *shape, seed=q, stream=3)
    x = fq.pack(q, to_dev(R))
    words, pad = packed_words(x)
    assert np.array_equal(words, encoding.pack(q, R))
    assert not pad.any()
    assert np.array_equal(fq.unpack(x).cpu().numpy(), R)


@pytest.mark.parametrize("q", EXT)
def test_pack_rejects_out_of_range_codes(fq, q):
    R = inputs.uniform(q, 3, 80, seed=1, stream=0)
    R[1, 7] = q
    R[2, 79] = 255
    x = fq.pack(q, to_dev(R))
    assert fq.status() == fq.EVALUE
    R[1, 7] = 0
    R[2, 79] = 0
    assert np.array_equal(fq.unpack(x).cpu().numpy(), R)


@pytest.mark.parametrize("q", EXT)
@pytest.mark.parametrize("sub", [False, True])
def test_add_sub_coefficientwise(fq, q, sub):
    p, n, _ = EXTENSIONS[q]
    X = inputs.uniform(q, 5, 300, seed=2, stream=0)
    Y = inputs.uniform(q, 5, 300, seed=2, stream=1)
    z = fq.add(fq.pack(q, to_dev(X)), fq.pack(q, to_dev(Y)), sub=sub)
    got = fq.unpack(z).cpu().numpy()
    sign = -1 if sub else 1
    want = oracle.compose(q, [(x.astype(np.int64) + sign * y.astype(np.int64)) % p
                              for x, y in zip(oracle.digits(q, X), oracle.digits(q, Y))])
    assert np.array_equal(got, want)
    if not sub:
        assert np.array_equal(got, pins.fadd(q, X, Y))


@pytest.mark.parametrize("q", EXT)
@pytest.mark.parametrize("mln", [(1, 1, 1), (3, 7, 5), (37, 100, 70), (300, 64, 1024), (513, 257, 1025)])
def test_product_matches_oracle(fq, q, mln):
    check(fq, q, *mln, seed=sum(mln) + q)


@pytest.mark.parametrize("q", EXT)
@pytest.mark.parametrize("path", ["m4rm", "mma"])
def test_base_products_on_each_path(fq, q, path):
    """The base-field products run on the requested path; both are exact."""
    check(fq, q, 260, 700, 530, seed=q, path=fq.PATH_M4RM if path == "m4rm" else fq.PATH_MMA)


@pytest.mark.parametrize("q", EXT)
def test_product_sparse_a(fq, q):
    check(fq, q, 400, 600, 300, seed=3, sparse=True)


@pytest.mark.parametrize("q", EXT)
def test_forced_base_kernel_and_block_size(fq, q):
    """k, rows per CTA and the compiled kernel index apply to the base field."""
    p = EXTENSIONS[q][0]
    check(fq, q, 200, 333, 130, seed=7, k=7)
    check(fq, q, 200, 333, 130, seed=8, variant=33)
    check(fq, q, 200, 333, 130, seed=9, kernel=len(fq.kernels(p)))


@pytest.mark.parametrize("q", EXT)
def test_identity_permutation_and_scalar(fq, q):
    n = 150
    B = inputs.uniform(q, n, 90, seed=1, stream=1)
    perm = np.random.default_rng(q).permutation(n)
    Pm = np.zeros((n, n), np.uint8)
    Pm[np.arange(n), perm] = 1
    got = fq.unpack(fq.matmul(fq.pack(q, to_dev(Pm)), fq.pack(q, to_dev(B)))).cpu().numpy()
    assert np.array_equal(got, B[perm])
    # x I times B multiplies every entry by the field element x (code p)
    xI = (np.eye(n, dtype=np.uint8) * EXTENSIONS[q][0]).astype(np.uint8)
    got = fq.unpack(fq.matmul(fq.pack(q, to_dev(xI)), fq.pack(q, to_dev(B)))).cpu().numpy()
    T = oracle.ext_mul_table(q)
    assert np.array_equal(got, T[EXTENSIONS[q][0], B.astype(np.int64)])


@pytest.mark.parametrize("q", EXT)
def test_degenerate_shapes(fq, q):
    c = fq.empty(q, 5, 70)
    c.data.fill_(-1)
    fq.matmul(fq.empty(q, 5, 0), fq.empty(q, 0, 70), out=c)
    assert not c.data.cpu().numpy().any()
    fq.matmul(fq.empty(q, 0, 9), fq.empty(q, 9, 4))
    fq.matmul(fq.empty(q, 3, 9), fq.empty(q, 9, 0))
    assert fq.status() == fq.OK


def test_gf4_three_f2_products(fq):
    """GF(4) by Section 4.3's three F_2 products equals the oracle and the
    elementwise GF(4) kernel, plane for plane."""
    for mln in ((1, 1, 1), (37, 100, 70), (513, 257, 1025), (1100, 520, 600)):
        c = check(fq, 4, *mln, seed=sum(mln), path=fq.PATH_KARATSUBA)
    A = inputs.uniform(4, 1536, 1536, seed=4, stream=inputs.STREAM_A)
    B = inputs.uniform(4, 1536, 1536, seed=4, stream=inputs.STREAM_B)
    a, b = fq.pack(4, to_dev(A)), fq.pack(4, to_dev(B))
    assert torch.equal(fq.matmul(a, b, path=fq.PATH_KARATSUBA).data, fq.matmul(a, b, path=fq.PATH_M4RM).data)


@pytest.mark.parametrize("q", (9, 125))
def test_graph_capture_of_an_extension_product(fq, q):
    """The stream-ordered scratch is captured as allocation nodes: replaying the
    graph recomputes the product into the same output."""
    A = inputs.uniform(q, 300, 400, seed=5, stream=inputs.STREAM_A)
    B = inputs.uniform(q, 400, 200, seed=5, stream=inputs.STREAM_B)
    a, b = fq.pack(q, to_dev(A)), fq.pack(q, to_dev(B))
    c = fq.empty(q, 300, 200)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        fq.matmul(a, b, out=c, stream=stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fq.matmul(a, b, out=c, stream=stream)
    c.data.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(fq.unpack(c).cpu().numpy(), oracle.matmul(q, A, B))
    assert fq.status() == fq.OK


@pytest.mark.slow
@pytest.mark.parametrize("q", EXT)
def test_product_1024_full_oracle(fq, q):
    check(fq, q, 1024, 1024, 1024, seed=q)


@pytest.mark.slow
@pytest.mark.parametrize("q", EXT)
def test_product_4096_sampled_rows_cols_and_freivalds(fq, q):
    """4096^3 over every extension field: 256 exact oracle rows and 256 exact
    oracle columns (the last of each among them) and a 32-trial Freivalds
    check (a wrong product passes with probability at most q^-32)."""
    n = 4096
    A = inputs.uniform(q, n, n, seed=1, stream=inputs.STREAM_A)
    B = inputs.uniform(q, n, n, seed=1, stream=inputs.STREAM_B)
    got = fq.unpack(fq.matmul(fq.pack(q, to_dev(A)), fq.pack(q, to_dev(B)))).cpu().numpy()
    assert fq.status() == fq.OK
    rng = np.random.default_rng(q)
    rows = np.unique(np.append(rng.choice(n, size=255, replace=False), n - 1))
    cols = np.unique(np.append(rng.choice(n, size=255, replace=False), n - 1))
    assert np.array_equal(got[rows], oracle.matmul_rows(q, A, B, rows))
    assert np.array_equal(got[:, cols], oracle.matmul_cols(q, A, B, cols))
    assert oracle.freivalds(q, A, B, got, trials=32, seed=q)
