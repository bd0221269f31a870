"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Integer work: every comparison is bit-exact (zero tolerance)."""
import ctypes
import itertools

import numpy as np
import pytest
import torch

import oracle
from oracle import encoding
from paper_0901_1413_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = (2, 3, 4, 5, 7)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def gpu_pack(fq, q, R):
    return fq.pack(q, to_dev(R))


def gpu_product(fq, q, A, B, **kw):
    a, b = gpu_pack(fq, q, A), gpu_pack(fq, q, B)
    c = fq.matmul(a, b, **kw)
    out = fq.unpack(c).cpu().numpy()
    assert fq.status() == fq.OK
    return out, c


def packed_words(x):
    """(planes, rows, ceil(cols/64)) uint64 from a Packed, plus its padding words."""
    v = x.planes_view().cpu().numpy().view(np.uint64)
    w = (x.cols + 63) // 64
    return v[:, :, :w], v[:, :, w:]


# ----------------------------------------------------------- pack / unpack --

@pytest.mark.parametrize("q", FIELDS)
@pytest.mark.parametrize("shape", [(1, 1), (3, 63), (5, 64), (7, 65), (33, 1000), (2, 1100)])
def test_pack_matches_oracle_encoding(fq, q, shape):
    R = inputs.uniform(q, *shape, seed=11, stream=q)
    x = gpu_pack(fq, q, R)
    words, pad = packed_words(x)
    assert np.array_equal(words, encoding.pack(q, R))
    assert not pad.any()
    assert np.array_equal(fq.unpack(x).cpu().numpy(), R)
    assert fq.status() == fq.OK


@pytest.mark.parametrize("q", FIELDS)
def test_pack_strided_and_unaligned_rows(fq, q):
    R = inputs.uniform(q, 9, 203, seed=3, stream=0)
    big = torch.zeros((9, 211), dtype=torch.uint8, device="cuda")
    big[:, 5:208] = to_dev(R)
    view = big[:, 5:208]                           # ld = 211, base not 16-byte aligned
    x = fq.pack(q, view)
    assert np.array_equal(packed_words(x)[0], encoding.pack(q, R))
    out = torch.full((9, 300), 255, dtype=torch.uint8, device="cuda")
    fq.unpack(x, out=out[:, 3:206])
    o = out.cpu().numpy()
    assert np.array_equal(o[:, 3:206], R)
    assert (o[:, :3] == 255).all() and (o[:, 206:] == 255).all()


@pytest.mark.parametrize("q", FIELDS)
def test_pack_rejects_out_of_range_residues(fq, q):
    R = inputs.uniform(q, 4, 100, seed=5, stream=0)
    R[2, 17] = q
    R[3, 99] = 200
    x = gpu_pack(fq, q, R)
    assert fq.status() == fq.EVALUE
    assert fq.status() == fq.OK                    # cleared
    R2 = R.copy()
    R2[2, 17] = 0
    R2[3, 99] = 0
    assert np.array_equal(fq.unpack(x).cpu().numpy(), R2)


@pytest.mark.parametrize("q", [5, 7])
def test_unpack_reduces_every_code(fq, q):
    """Any 3-bit code is read mod p (Section 4.2: codes are not unique)."""
    codes = np.arange(64, dtype=np.uint8) % 8
    planes = np.zeros((3, 1, 16), np.uint64)
    for p in range(3):
        planes[p, 0, 0] = np.uint64(sum(int((c >> p) & 1) << j for j, c in enumerate(codes)))
    x = fq.empty(q, 1, 64)
    x.data.copy_(torch.from_numpy(planes.reshape(-1).view(np.int64)))
    assert np.array_equal(fq.unpack(x).cpu().numpy()[0], codes % q)


# ---------------------------------------- bitsliced add/sub, every code pair --

def _code_planes(q, codes):
    P = encoding.planes(q)
    pl = np.zeros((P, 1, 16), np.uint64)
    for p in range(P):
        pl[p, 0, 0] = np.uint64(sum(int((int(c) >> p) & 1) << j for j, c in enumerate(codes)))
    return pl


def _value(q, code):
    if q == 3:
        return {0: 0, 1: 1, 3: 2}[code]
    return code % q if q != 4 else code


@pytest.mark.parametrize("q", FIELDS)
@pytest.mark.parametrize("sub", [False, True])
def test_add_sub_every_code_pair(fq, q, sub):
    codes = {2: [0, 1], 3: [0, 1, 3], 4: list(range(4))}.get(q, list(range(8)))
    pairs = list(itertools.product(codes, repeat=2))
    assert len(pairs) <= 64
    X = fq.empty(q, 1, 64)
    Y = fq.empty(q, 1, 64)
    X.data.copy_(torch.from_numpy(_code_planes(q, [a for a, _ in pairs]).reshape(-1).view(np.int64)))
    Y.data.copy_(torch.from_numpy(_code_planes(q, [b for _, b in pairs]).reshape(-1).view(np.int64)))
    Z = fq.add(X, Y, sub=sub)
    got = fq.unpack(Z).cpu().numpy()[0, :len(pairs)]
    for (a, b), g in zip(pairs, got):
        va, vb = _value(q, a), _value(q, b)
        if q == 4:
            want = va ^ vb
        else:
            want = (va - vb) % q if sub else (va + vb) % q
        assert g == want, (a, b)
    if q == 3:   # F_3 codes stay valid: never (x0, x1) = (0, 1)
        w = Z.planes_view().cpu().numpy().view(np.uint64)[:, 0, 0]
        assert int(~w[0] & w[1] & np.uint64((1 << len(pairs)) - 1)) == 0


# -------------------------------------------------------------- products --

def _check_product(fq, q, m, l, n, seed, sparse=False, **kw):
    A = (inputs.sparse if sparse else inputs.uniform)(q, m, l, seed=seed, stream=inputs.STREAM_A)
    B = inputs.uniform(q, l, n, seed=seed, stream=inputs.STREAM_B)
    got, c = gpu_product(fq, q, A, B, **kw)
    want = oracle.matmul(q, A, B)
    assert np.array_equal(got, want), "first mismatch at %s" % (np.argwhere(got != want)[:3].tolist(),)
    # output planes are canonical codes with zero padding
    words, pad = packed_words(c)
    assert np.array_equal(words, encoding.pack(q, want))
    assert not pad.any()
    return got, c


def test_config1_f3_512(fq):
    """F_3, A and B 512 x 512 uniform, k = 8, basis {1, -1}."""
    _check_product(fq, 3, 512, 512, 512, seed=0, k=8)


@pytest.mark.parametrize("q", FIELDS)
@pytest.mark.parametrize("mln", [(1, 1, 1), (3, 7, 5), (37, 100, 70), (300, 64, 1024),
                                 (513, 257, 1025), (1100, 520, 600)])
def test_product_matches_oracle(fq, q, mln):
    _check_product(fq, q, *mln, seed=sum(mln) + q)


@pytest.mark.parametrize("q", FIELDS)
def test_product_sparse_a(fq, q):
    _check_product(fq, q, 700, 900, 600, seed=9, sparse=True)


@pytest.mark.parametrize("q", FIELDS)
def test_product_all_max_closed_form(fq, q):
    """A, B filled with q-1: every entry is l (q-1)^2 mod q (GF(4): (alpha+1)^2 = alpha
    summed l times)."""
    m, l, n = 70, 1001, 130
    A = np.full((m, l), q - 1, np.uint8)
    B = np.full((l, n), q - 1, np.uint8)
    got, _ = gpu_product(fq, q, A, B)
    if q == 4:
        want = 2 if l % 2 else 0
    else:
        want = (l * (q - 1) ** 2) % q
    assert (got == want).all()


@pytest.mark.parametrize("q", FIELDS)
def test_product_degenerate_shapes(fq, q):
    # l = 0: C = 0
    a = fq.empty(q, 5, 0)
    b = fq.empty(q, 0, 70)
    c = fq.empty(q, 5, 70)
    c.data.fill_(-1)
    fq.matmul(a, b, out=c)
    assert not fq.unpack(c).cpu().numpy().any()
    assert not c.data.cpu().numpy().any()
    # m = 0 and n = 0 are no-ops
    fq.matmul(fq.empty(q, 0, 9), fq.empty(q, 9, 4))
    fq.matmul(fq.empty(q, 3, 9), fq.empty(q, 9, 0))
    assert fq.status() == fq.OK


@pytest.mark.parametrize("q", FIELDS)
def test_identity_and_permutation(fq, q):
    n = 300
    B = inputs.uniform(q, n, 200, seed=1, stream=1)
    perm = np.random.default_rng(q).permutation(n)
    Pm = np.zeros((n, n), np.uint8)
    Pm[np.arange(n), perm] = 1
    got, _ = gpu_product(fq, q, Pm, B)
    assert np.array_equal(got, B[perm])


@pytest.mark.parametrize("q,k", [(2, 6), (2, 7), (2, 9), (2, 10), (3, 6), (3, 7), (3, 9), (3, 10),
                                 (4, 6), (4, 9), (4, 10), (5, 6), (5, 7), (7, 6), (7, 7)])
def test_every_block_size(fq, q, k):
    """k = 6, 7, 9, 10 do not divide 64: indices straddle A's words."""
    _check_product(fq, q, 333, 777, 600, seed=k, k=k)


@pytest.mark.parametrize("q", FIELDS)
@pytest.mark.parametrize("mt", [1, 5, 33, 200])
def test_forced_rows_per_cta(fq, q, mt):
    """Tiles of any height, including partial row slots."""
    _check_product(fq, q, 410, 300, 520, seed=mt, variant=mt)


@pytest.mark.parametrize("q,kmax", [(3, 10), (5, 8)])
def test_unsupported_block_size_is_reported(fq, q, kmax):
    a = fq.empty(q, 4, 4)
    b = fq.empty(q, 4, 4)
    a.data.zero_()
    b.data.zero_()
    if kmax < 10:
        with pytest.raises(fq.FqError) as e:
            fq.matmul(a, b, k=kmax + 1)
        assert e.value.status == fq.ENOTSUP
    with pytest.raises(fq.FqError) as e:
        fq.matmul(a, b, variant=100000)
    assert e.value.status == fq.EINVAL


@pytest.mark.parametrize("q", [2, 3, 4, 5, 7])
@pytest.mark.parametrize("k", [6, 7, 9])
def test_last_block_reaches_past_the_pitch(fq, q, k):
    """l = 1024 is a whole pitch: with k not dividing 64 the last block's index
    field extends past the row's last word."""
    if q in (5, 7) and k == 9:
        pytest.skip("three-plane tables stop at k = 8")
    _check_product(fq, q, 200, 1024, 130, seed=k, k=k)


@pytest.mark.parametrize("q", FIELDS)
def test_every_compiled_kernel(fq, q):
    """Each compiled M4RM kernel (block size, tile shape, warp layout) on a ragged
    product, bit-exact against the oracle."""
    ks = fq.kernels(q)
    assert len(ks) >= 5
    A = inputs.uniform(q, 333, 777, seed=q, stream=inputs.STREAM_A)
    B = inputs.uniform(q, 777, 600, seed=q, stream=inputs.STREAM_B)
    want = oracle.matmul(q, A, B)
    a, b = gpu_pack(fq, q, A), gpu_pack(fq, q, B)
    for info in ks:
        got = fq.unpack(fq.matmul(a, b, kernel=info["index"] + 1)).cpu().numpy()
        assert np.array_equal(got, want), info
    assert fq.status() == fq.OK


# ------------------------------------------------ exact tensor-core path --

@pytest.mark.parametrize("q", FIELDS)
@pytest.mark.parametrize("mln", [(1, 1, 1), (37, 100, 70), (300, 500, 260), (513, 257, 1025)])
def test_mma_path_matches_oracle(fq, q, mln):
    _check_product(fq, q, *mln, seed=sum(mln) + 7 * q, path=fq.PATH_MMA)


@pytest.mark.parametrize("q", FIELDS)
@pytest.mark.parametrize("mln", [(1, 1, 1), (37, 100, 70), (300, 500, 260), (513, 257, 1025)])
def test_mma_sync_form_matches_oracle(fq, q, mln):
    """The mma.sync s8 form (fq_options.kernel = 1), kept for l beyond the
    tcgen05 form's exact range."""
    _check_product(fq, q, *mln, seed=sum(mln) + 11 * q, path=fq.PATH_MMA, kernel=1)


@pytest.mark.parametrize("kernel", [2, 3, 4, 5])
@pytest.mark.parametrize("q", FIELDS)
@pytest.mark.parametrize("mln", [(1, 1, 1), (128, 300, 257), (129, 300, 257), (300, 500, 260), (513, 257, 1025),
                                 (260, 1300, 1100)])
def test_tcgen05_forms_match_oracle(fq, q, mln, kernel):
    """fq_options.kernel = 2, 3, 4, 5: the single-SM tcgen05 kernel (128 x 256
    tiles), the SM-pair kernel (256 x 256) and the wide SM-pair kernel (256 x
    512) from e4m3 operands, and the SM-pair kernel from packed e2m1 operands
    (kind::mxf4, 256 x 448 tiles), each forced whatever the shape; equal to
    the oracle and to the form the shape takes by default."""
    got, c1 = _check_product(fq, q, *mln, seed=sum(mln) + 13 * q, path=fq.PATH_MMA, kernel=kernel)
    m, l, n = mln
    A = inputs.uniform(q, m, l, seed=sum(mln) + 13 * q, stream=inputs.STREAM_A)
    B = inputs.uniform(q, l, n, seed=sum(mln) + 13 * q, stream=inputs.STREAM_B)
    c0 = fq.matmul(gpu_pack(fq, q, A), gpu_pack(fq, q, B), path=fq.PATH_MMA)
    assert torch.equal(c0.data, c1.data)


@pytest.mark.parametrize("group", [1, 3, 64])
def test_tcgen05_tile_order_groups(fq, group):
    """fq_options.variant on the tcgen05 path sets the tile order's row-block
    group; every order gives the same, exact product (ragged m and n)."""
    _check_product(fq, 3, 1100, 300, 2100, seed=group, path=fq.PATH_MMA, variant=group)
    _check_product(fq, 5, 700, 200, 1500, seed=group, path=fq.PATH_MMA, variant=group, kernel=2)


@pytest.mark.parametrize("q", FIELDS)
def test_tensor_operands_prepared_once(fq, q):
    """fq_tc_prepare once, fq_tc_multiply twice: both results equal the oracle."""
    m, l, n = 300, 520, 700
    A = inputs.uniform(q, m, l, seed=q + 60, stream=inputs.STREAM_A)
    B = inputs.uniform(q, l, n, seed=q + 60, stream=inputs.STREAM_B)
    ops = fq.TensorOperands(gpu_pack(fq, q, A), gpu_pack(fq, q, B))
    want = oracle.matmul(q, A, B)
    c1 = ops.multiply()
    c2 = ops.multiply()
    assert np.array_equal(fq.unpack(c1).cpu().numpy(), want)
    assert torch.equal(c1.data, c2.data)
    assert fq.status() == fq.OK


# Every tcgen05 product kernel: (rows, forced kernel) -- single SMs, the two
# e4m3 SM-pair forms and the fp4 SM-pair form (rows 260: the second half of
# the pair's row block lies outside m).
TC_KERNELS = [(3, 2), (260, 3), (260, 4), (260, 5)]


@pytest.mark.slow
@pytest.mark.parametrize("m, kernel", TC_KERNELS)
def test_tcgen05_exact_near_its_range(fq, m, kernel):
    """F_7 with every entry 3: each entry of C is 9 l before the reduction,
    9.4e6 for l = 2^20 (the fp32 sums must stay exact up to 2^24)."""
    l, n = 1 << 20, 70
    A = np.full((m, l), 3, np.uint8)
    B = np.full((l, n), 3, np.uint8)
    got, _ = gpu_product(fq, 7, A, B, path=fq.PATH_MMA, kernel=kernel)
    assert (got == (9 * l) % 7).all()


@pytest.mark.slow
@pytest.mark.parametrize("m, kernel", TC_KERNELS)
@pytest.mark.parametrize("q, l, codes", [(7, None, (1, 2, 3)), (5, None, (1, 2)), (3, 1 << 22, (0, 1))])
def test_tcgen05_exact_with_random_low_bits(fq, q, l, codes, m, kernel):
    """Rows of A all +3 (F_7), +2 (F_5) or +1 (F_3) against random positive B:
    every step of the tensor-core sum adds a random amount, so an
    accumulation that dropped low bits anywhere on the way to 2^24 (F_7 and
    F_5 at their longest exact l) or 2^22 (F_3) would change the residues.
    C = A B is a column sum of B.  Every product kernel, e4m3 and packed e2m1
    (block scale factors 1.0)."""
    l = l or _tc_max_l(fq, q)
    n = 70
    a = {7: 3, 5: 2, 3: 1}[q]
    A = np.full((m, l), a, np.uint8)
    B = np.random.default_rng(q).choice(np.array(codes, np.uint8), size=(l, n))
    got, _ = gpu_product(fq, q, A, B, path=fq.PATH_MMA, kernel=kernel)
    want = (a * B.sum(axis=0, dtype=np.int64)) % q
    assert (got == want[None, :]).all()


SMALL_SUM = (1 << 22) - 8   # the epilogue's one-add conversion covers |sum| <= 2^22 - 8


@pytest.mark.slow
@pytest.mark.parametrize("m, kernel", [(3, 2), (260, 5)])
@pytest.mark.parametrize("q, a, top", [(3, 1, 1), (3, 2, 1), (5, 2, 2), (5, 3, 2), (7, 3, 3), (7, 4, 3)])
@pytest.mark.parametrize("extra", [0, 1])
def test_tcgen05_sums_at_the_epilogue_boundary(fq, q, a, top, m, kernel, extra):
    """Every row of A is a (balanced +-top) and column 0 of B is all +top,
    column 1 all -top, so the two sums are +-l top^2: exactly +-(2^22 - 8) at
    the longest l whose sums the epilogue reads through one add, and one term
    past it (extra = 1), where it reads them through the truncating
    conversion; the other columns are random.  C = a colsum(B) mod q."""
    l = SMALL_SUM // (top * top) + extra
    n = 70
    A = np.full((m, l), a, np.uint8)
    B = np.random.default_rng(l + q).integers(0, q, size=(l, n), dtype=np.uint8)
    B[:, 0] = top
    B[:, 1] = q - top
    got, _ = gpu_product(fq, q, A, B, path=fq.PATH_MMA, kernel=kernel)
    want = (a * B.sum(axis=0, dtype=np.int64)) % q
    assert (got == want[None, :]).all()


@pytest.mark.parametrize("q", FIELDS)
@pytest.mark.parametrize("k", range(1, 8))
def test_fp4_form_every_last_tile_width(fq, q, k):
    """The fp4 SM-pair form's column tiles are 448 wide; the last one takes
    what is left of the 1024 k-column pitch: 128, 256, 384, 64, 192, 320 and
    448 for k = 1 .. 7 (two MMA halves of up to 224 columns, the second one
    narrower or absent).  n = 1024 k - 100 leaves padding columns too."""
    _check_product(fq, q, 300, 600, 1024 * k - 100, seed=40 + k, path=fq.PATH_MMA, kernel=5)


def _tc_max_l(fq, q):
    """Longest l the tcgen05 form takes for q (found through the workspace query)."""
    lib = fq.load()
    lo, hi = 1, 1 << 26
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if lib.fq_tc_workspace_bytes(q, 1, mid, 1) >= 0:
            lo = mid
        else:
            hi = mid - 1
    return lo


@pytest.mark.parametrize("q", FIELDS)
@pytest.mark.parametrize("chunk", [64, 128, 1000])
def test_mma_path_reduces_between_chunks(fq, q, chunk):
    """A forced short l-chunk runs the mod-p reduction between chunks many times."""
    _check_product(fq, q, 130, 1100, 200, seed=chunk, path=fq.PATH_MMA, chunk=chunk)


@pytest.mark.parametrize("q", FIELDS)
def test_mma_path_all_max(fq, q):
    m, l, n = 70, 3001, 130
    A = np.full((m, l), q - 1, np.uint8)
    B = np.full((l, n), q - 1, np.uint8)
    got, _ = gpu_product(fq, q, A, B, path=fq.PATH_MMA, chunk=64)
    want = (2 if l % 2 else 0) if q == 4 else (l * (q - 1) ** 2) % q
    assert (got == want).all()


@pytest.mark.parametrize("q", FIELDS)
def test_paths_agree_bit_for_bit(fq, q):
    """M4RM and the tensor-core form give identical planes."""
    n = 1536
    A = inputs.uniform(q, n, n, seed=q, stream=inputs.STREAM_A)
    B = inputs.uniform(q, n, n, seed=q, stream=inputs.STREAM_B)
    a, b = gpu_pack(fq, q, A), gpu_pack(fq, q, B)
    c1 = fq.matmul(a, b, path=fq.PATH_M4RM)
    c2 = fq.matmul(a, b, path=fq.PATH_MMA)
    assert torch.equal(c1.data, c2.data)
    assert fq.status() == fq.OK


def test_mma_path_degenerate(fq):
    c = fq.empty(5, 4, 70)
    c.data.fill_(-1)
    fq.matmul(fq.empty(5, 4, 0), fq.empty(5, 0, 70), out=c, path=fq.PATH_MMA)
    assert not c.data.cpu().numpy().any()


@pytest.mark.parametrize("q", FIELDS)
def test_autotune_picks_a_candidate_and_auto_uses_it(fq, q):
    lib = fq.load()
    lib.fq_autotune_clear()
    m, l, n = 700, 900, 600
    A = inputs.uniform(q, m, l, seed=21, stream=inputs.STREAM_A)
    B = inputs.uniform(q, l, n, seed=21, stream=inputs.STREAM_B)
    a, b = gpu_pack(fq, q, A), gpu_pack(fq, q, B)
    c = fq.empty(q, m, n)
    res = fq.autotune(a, b, out=c)
    want = oracle.matmul(q, A, B)
    assert np.array_equal(fq.unpack(c).cpu().numpy(), want)          # C holds the product
    assert res["path"] in (fq.PATH_M4RM, fq.PATH_MMA) and res["ms"] > 0
    assert res["ms"] <= res["ms_planner"] + 1e-6 and res["ms"] <= res["ms_mma"] + 1e-6
    path, kernel = ctypes.c_int(), ctypes.c_int()
    assert lib.fq_autotune_lookup(q, m, l, n, ctypes.byref(path), ctypes.byref(kernel)) == fq.OK
    assert (path.value, kernel.value) == (res["path"], res["kernel"])
    got = fq.unpack(fq.matmul(a, b)).cpu().numpy()                       # AUTO: the tuned choice
    assert np.array_equal(got, want)
    if res["path"] == fq.PATH_M4RM and res["kernel"] > 0:
        assert fq.planned_kernel(q, m, l, n)["index"] == res["kernel"] - 1
    lib.fq_autotune_clear()
    assert lib.fq_autotune_lookup(q, m, l, n, None, None) == fq.ENOTSUP


def test_auto_choice_by_time_model(fq):
    """Without a measurement, AUTO takes the tcgen05 tensor-core path for every
    base field at 8192^3 (measured on GB300: F_3 0.40 vs 1.53 ms, F_2 0.37 vs
    0.74 ms, GF(4)'s three F_2 products about 1.2 vs 1.34 ms); empty products
    take the M4RM planner; all give the oracle's result."""
    fq.load().fq_autotune_clear()
    assert fq.auto_choice(3, 512, 512, 512) == (fq.PATH_MMA, 0)
    for q in FIELDS:
        assert fq.auto_choice(q, 8192, 8192, 8192) == (fq.PATH_MMA, 0)
    assert fq.auto_choice(3, 0, 512, 512) == (fq.PATH_M4RM, 0)
    for q in FIELDS:
        _check_product(fq, q, 512, 512, 512, seed=q + 40)       # AUTO, whichever path


@pytest.mark.parametrize("q", FIELDS)
def test_planned_kernel_honours_k(fq, q):
    for k in (6, 7, 8):
        assert fq.planned_kernel(q, 3000, 2000, 4000, k=k)["k"] == k


@pytest.mark.parametrize("q", FIELDS)
def test_auto_choice_follows_autotune(fq, q):
    lib = fq.load()
    lib.fq_autotune_clear()
    a, b = fq.empty(q, 300, 200), fq.empty(q, 200, 100)
    a.data.zero_()
    b.data.zero_()
    res = fq.autotune(a, b)
    assert fq.auto_choice(q, 300, 200, 100) == (res["path"], res["kernel"])
    lib.fq_autotune_clear()
