"""The CPU oracle, pinned by checks that do not restate its own formula."""
import os

import numpy as np
import pytest

import ctypes

import oracle
from oracle import encoding, m4rm
from oracle.fields import EXTENSIONS
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FIELDS = oracle.FIELDS
BASE_FIELDS = (2, 3, 4, 5, 7)


def run_pins(mm, q):
    return pins.run_all(mm, q, seed=q, karatsuba=oracle.gf4_karatsuba, ext_karatsuba=oracle.ext_karatsuba)


@pytest.mark.parametrize("q", FIELDS)
def test_oracle_passes_all_pins(q):
    assert run_pins(oracle.matmul, q) == []


# --- planted mistakes: each mutant of the oracle must fail at least one pin ---

def _mut_dropped_term(q, A, B):          # the last term a_{i,l-1} B_{l-1} is lost
    A = np.array(A, copy=True)
    if A.shape[1]:
        A[:, -1] = 0
    return oracle.matmul(q, A, B)


def _mut_wrong_index(q, A, B):           # row j of B paired with a_{i,j+1}
    return oracle.matmul(q, A, np.ascontiguousarray(np.roll(B, 1, axis=0)))


def _mut_transposed(q, A, B):            # A^T B whenever the shapes allow it
    if A.shape[0] == A.shape[1]:
        return oracle.matmul(q, np.ascontiguousarray(A.T), B)
    return oracle.matmul(q, A, B)


def _mut_sign(q, A, B):                  # first term subtracted instead of added
    C = oracle.matmul(q, A, B).astype(np.int64)
    if q == 4 or q == 8:
        return C.astype(np.uint8)            # (char 2: -x = x, no sign to flip)
    if q in EXTENSIONS:
        p = EXTENSIONS[q][0]
        first = oracle.matmul(q, np.ascontiguousarray(A[:, :1]), np.ascontiguousarray(B[:1])) \
            if A.shape[1] else np.zeros_like(C)
        c, f = oracle.digits(q, C), oracle.digits(q, first)
        return oracle.compose(q, [(x.astype(np.int64) - 2 * y) % p for x, y in zip(c, f)])
    first = np.outer(A[:, 0].astype(np.int64), B[0].astype(np.int64)) if A.shape[1] else 0
    return ((C - 2 * first) % q).astype(np.uint8)


def _mut_narrow_accumulator(q, A, B):    # int8-wide accumulation that wraps
    if q in EXTENSIONS:
        return oracle.matmul(q, A, B)
    acc = (A.astype(np.uint8) @ B.astype(np.uint8)).astype(np.uint8)
    return (acc % q).astype(np.uint8)


def _mut_gf4_wrong_poly(q, A, B):        # GF(4) reduced with x^2 = 1 instead of x + 1
    if q != 4:
        return oracle.matmul(q, A, B)
    A0, A1 = A & 1, (A >> 1) & 1
    B0, B1 = B & 1, (B >> 1) & 1
    e0 = oracle.matmul(2, A0, B0) ^ oracle.matmul(2, A1, B1)
    e1 = oracle.matmul(2, A0, B1) ^ oracle.matmul(2, A1, B0)
    return (e0 | (e1 << 1)).astype(np.uint8)


def _mut_ext_wrong_poly(q, A, B):       # reduced with r_0 + 1 in place of r_0
    if q not in EXTENSIONS:
        return oracle.matmul(q, A, B)
    p, n, r = EXTENSIONS[q]
    bad = list(r)
    bad[0] = (bad[0] + 1) % p
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    C = np.zeros((A.shape[0], B.shape[1]), np.uint8)
    u8 = lambda X: X.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    rc = oracle._load().fq_oracle_matmul_ext(p, n, (ctypes.c_int * n)(*bad), A.shape[0], A.shape[1], B.shape[1],
                                             u8(A), A.shape[1], u8(B), B.shape[1], u8(C), B.shape[1], 1)
    assert rc == 0
    return C


MUTANTS = {
    "dropped_term": _mut_dropped_term,
    "wrong_index": _mut_wrong_index,
    "transposed": _mut_transposed,
    "sign": _mut_sign,
    "narrow_accumulator": _mut_narrow_accumulator,
    "gf4_wrong_poly": _mut_gf4_wrong_poly,
    "ext_wrong_poly": _mut_ext_wrong_poly,
}


@pytest.mark.parametrize("q", FIELDS)
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistakes(q, name):
    if (q in EXTENSIONS and name == "narrow_accumulator") or (q != 4 and name == "gf4_wrong_poly") \
            or (q not in EXTENSIONS and name == "ext_wrong_poly"):
        pytest.skip("mutant is the identity for this field")
    if q in (2, 4, 8) and name == "sign":
        pytest.skip("char 2: -x = x")
    if q == 2 and name == "narrow_accumulator":
        pytest.skip("a wrap mod 256 preserves parity: the mutant is correct over F_2")
    fails = run_pins(MUTANTS[name], q)
    assert fails, "mutant %s survived every pin for q=%d" % (name, q)


# --- the paper's method, step by step, reaches the plain product ---

@pytest.mark.parametrize("q", BASE_FIELDS)
@pytest.mark.parametrize("k", [1, 3, 4, 8])
def test_m4rm_method_matches_plain_product(q, k):
    rng = np.random.default_rng(100 + q * 10 + k)
    m, l, n = 9, 23, 70                      # k does not divide l; n spans two words
    A, B = pins.rand(rng, q, m, l), pins.rand(rng, q, l, n)
    assert np.array_equal(m4rm.m4rm(q, A, B, k), oracle.matmul(q, A, B))


def test_m4rm_method_zero_and_degenerate():
    A = np.zeros((4, 5), np.uint8)
    B = np.zeros((5, 3), np.uint8)
    assert not m4rm.m4rm(3, A, B, 2).any()
    assert m4rm.m4rm(5, np.zeros((0, 5), np.uint8), B, 2).shape == (0, 3)


# --- GF(4): the two oracles agree; brute force over every 2x2 product ---

def test_gf4_karatsuba_agrees_with_polynomial_oracle():
    rng = np.random.default_rng(4)
    for m, l, n in ((1, 1, 1), (17, 65, 31), (64, 128, 64)):
        A, B = pins.rand(rng, 4, m, l), pins.rand(rng, 4, l, n)
        assert np.array_equal(oracle.matmul(4, A, B), oracle.gf4_karatsuba(A, B))


@pytest.mark.parametrize("q", [3, 4])
def test_brute_force_all_2x2_products(q):
    """Every pair of 2x2 matrices (q^8 products) against the Section 4.3
    Karatsuba form (GF(4)) or numpy (F_3), batched as one block-diagonal product."""
    vals = np.array(np.meshgrid(*[np.arange(q)] * 4, indexing="ij")).reshape(4, -1).T.astype(np.uint8)
    mats = vals.reshape(-1, 2, 2)
    N = len(mats)
    Astack = np.repeat(mats, N, axis=0)          # pair (a, b) -> A = mats[a], B = mats[b]
    Bstack = np.tile(mats, (N, 1, 1))
    # one product per pair: rows of A_pair against B_pair, computed pair by pair in bulk
    # by the oracle on a (2, 2) x (2, 2N^2)-wide layout per A
    got = np.empty_like(Astack)
    for a in range(N):
        Bwide = np.ascontiguousarray(np.concatenate(list(Bstack[a * N:(a + 1) * N]), axis=1))
        got[a * N:(a + 1) * N] = oracle.matmul(q, mats[a], Bwide).reshape(2, N, 2).transpose(1, 0, 2)
    if q == 3:
        ref = np.einsum("pij,pjk->pik", Astack.astype(np.int64), Bstack.astype(np.int64)) % 3
    else:
        ref = np.stack([oracle.gf4_karatsuba(x, y) for x, y in zip(Astack[::97], Bstack[::97])])
        got = got[::97]
    assert np.array_equal(got, ref)


# --- extension fields: the two oracles, the polynomials, the codes ---

def test_extension_oracle_equals_gf4_oracle():
    """The tabulated extension-field oracle at (p, n) = (2, 2) and the separate
    GF(4) routine are independent codes for the same field."""
    rng = np.random.default_rng(44)
    for m, l, n in ((1, 1, 1), (19, 67, 33), (64, 130, 64)):
        A, B = pins.rand(rng, 4, m, l), pins.rand(rng, 4, l, n)
        assert np.array_equal(oracle.matmul_ext(4, A, B), oracle.matmul(4, A, B))


@pytest.mark.parametrize("q", sorted(EXTENSIONS))
def test_defining_polynomial_of_x(q):
    """x^n in the oracle's arithmetic is r_0 + r_1 x + ... (the stated
    polynomial), and no lower power of x reduces (x^j has code p^j, j < n)."""
    p, n, r = EXTENSIONS[q]
    T = pins.mul_table(oracle.matmul, q)
    y = 1
    for j in range(n):
        assert y == p ** j
        y = int(T[y, p])
    assert y == sum(c * p ** j for j, c in enumerate(r))


@pytest.mark.parametrize("q", sorted(EXTENSIONS))
def test_extension_codes_round_trip(q):
    rng = np.random.default_rng(q)
    R = pins.rand(rng, q, 7, 130)
    planes = encoding.pack(q, R)
    assert planes.shape == (encoding.planes(q), 7, 3)
    assert np.array_equal(encoding.unpack(q, planes, 130), R)
    p, n, _ = EXTENSIONS[q]
    P = encoding.planes(p)
    for j, d in enumerate(oracle.digits(q, R)):           # coefficient j's planes
        assert np.array_equal(planes[j * P:(j + 1) * P], encoding.pack(p, d))


# --- checks used at sizes the full oracle cannot reach ---

@pytest.mark.parametrize("q", FIELDS)
def test_randomized_check_products_equal_the_oracle(q):
    """The exact product the randomized check uses (float64 library matmul by
    row chunks; polynomial coefficients for extension fields) equals the C
    oracle's row combination, with chunks of one row and of several rows."""
    rng = np.random.default_rng(70 + q)
    M = pins.rand(rng, q, 37, 53)
    X = pins.rand(rng, q, 53, 11)
    want = oracle.matmul(q, M, X)
    for chunk in (1, 8 * 53 * 5, 1 << 28):
        got = oracle._field_matmul(q, M, X.astype(np.int64), chunk_bytes=chunk)
        assert got.dtype == np.int64
        assert np.array_equal(got, want)


@pytest.mark.parametrize("q", FIELDS)
def test_freivalds_accepts_product_and_rejects_one_wrong_entry(q):
    rng = np.random.default_rng(7)
    A, B = pins.rand(rng, q, 40, 50), pins.rand(rng, q, 50, 30)
    C = oracle.matmul(q, A, B)
    assert oracle.freivalds(q, A, B, C, trials=32)
    assert oracle.freivalds(q, A, B, C, trials=32, chunk_bytes=8 * 50 * 3)
    for (i, j) in ((0, 0), (13, 17), (39, 29)):
        for delta in range(1, q):
            bad = C.copy()
            bad[i, j] = (int(bad[i, j]) + delta) % q
            assert not oracle.freivalds(q, A, B, bad, trials=32, chunk_bytes=8 * 50 * 3)


@pytest.mark.parametrize("q", [2, 3])
def test_freivalds_trials_are_independent(q):
    """One wrong entry e at (i, j): a trial passes exactly when x_j = 0, with
    probability 1/q, so over many seeds t trials pass about q^-t of the time
    (a check whose vectors were fixed or not uniform would pass always or never)."""
    rng = np.random.default_rng(11)
    A, B = pins.rand(rng, q, 12, 10), pins.rand(rng, q, 10, 9)
    bad = oracle.matmul(q, A, B)
    bad[4, 5] = (int(bad[4, 5]) + 1) % q
    seeds = range(600)
    for t in (1, 2):
        passed = sum(oracle.freivalds(q, A, B, bad, trials=t, seed=s) for s in seeds)
        expect = len(seeds) / q ** t
        assert abs(passed - expect) < 5 * (expect * (1 - q ** -t)) ** 0.5, (t, passed, expect)


def test_freivalds_refuses_sums_beyond_float64():
    """Sums of l products of at most (p - 1)^2 are exact float64 integers only
    while l (p - 1)^2 < 2^53: longer rows are refused (a broadcast view has the
    shape without the memory)."""
    wide = np.broadcast_to(np.zeros(1, np.uint8), (1, 1 << 48))
    with pytest.raises(ValueError):
        oracle._fp_matmul(7, wide, np.zeros((1, 1), np.int64))
    ok = np.broadcast_to(np.zeros(1, np.uint8), (1, 3))
    assert oracle._fp_matmul(7, ok, np.ones((3, 1), np.int64)).tolist() == [[0]]


@pytest.mark.parametrize("q", [5, 4, 9])
def test_matmul_rows_and_cols_are_slices(q):
    rng = np.random.default_rng(8)
    A, B = pins.rand(rng, q, 30, 20), pins.rand(rng, q, 20, 10)
    C = oracle.matmul(q, A, B)
    rows, cols = [0, 7, 29], [9, 0, 4, 4]
    assert np.array_equal(oracle.matmul_rows(q, A, B, rows), C[rows])
    assert np.array_equal(oracle.matmul_cols(q, A, B, cols), C[:, cols])


def test_thread_count_does_not_change_result():
    rng = np.random.default_rng(9)
    A, B = pins.rand(rng, 7, 100, 90), pins.rand(rng, 7, 90, 80)
    assert np.array_equal(oracle.matmul(7, A, B, threads=1), oracle.matmul(7, A, B, threads=4))
    assert oracle.threads_used(3) == 3


def test_oracle_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.matmul(6, np.zeros((2, 2), np.uint8), np.zeros((2, 2), np.uint8))
    with pytest.raises(ValueError):
        oracle.matmul(3, np.full((2, 2), 3, np.uint8), np.zeros((2, 2), np.uint8))
    with pytest.raises(ValueError):
        oracle.matmul(3, np.zeros((2, 3), np.uint8), np.zeros((2, 2), np.uint8))


def test_empty_dimensions():
    for m, l, n in ((0, 5, 3), (4, 0, 3), (4, 5, 0)):
        C = oracle.matmul(3, np.zeros((m, l), np.uint8), np.zeros((l, n), np.uint8))
        assert C.shape == (m, n) and not C.any()


# --- the representation (Sections 3 and 4.1) ---

def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_worked_example_planes_section3():
    g = {r[0]: r[1:] for r in _read_golden("z4_worked_example.txt")}
    values = np.array([int(v) for v in g["values"]], np.uint8)
    # Z/4 codes are the values' binary digits; use the generic binary planes.
    bits = [(values >> i) & 1 for i in range(2)]
    display = lambda b: "".join(str(int(x)) for x in b)   # element 0 at the left
    assert display(bits[1]) == g["plane1"][0]
    assert display(bits[0]) == g["plane0"][0]
    words = encoding._bits_to_words(np.stack(bits))
    assert encoding._words_to_bits(words, 8).tolist() == [list(b) for b in bits]


def test_f3_representation_section41():
    for value, code in _read_golden("f3_representation.txt"):
        x0, x1 = encoding.codes_to_bits(3, np.array([int(value)]))
        assert "%d%d" % (x0[0], x1[0]) == code


@pytest.mark.parametrize("q", FIELDS)
def test_pack_unpack_round_trip(q):
    rng = np.random.default_rng(q)
    for r, c in ((1, 1), (3, 64), (5, 65), (7, 200)):
        R = pins.rand(rng, q, r, c)
        Pl = encoding.pack(q, R)
        assert Pl.shape == (encoding.planes(q), r, (c + 63) // 64)
        assert np.array_equal(encoding.unpack(q, Pl, c), R)


def test_pack_bit_order():
    R = np.zeros((1, 130), np.uint8)
    R[0, 0] = 1
    R[0, 65] = 2
    R[0, 129] = 1
    Pl = encoding.pack(3, R)
    assert Pl[0, 0].tolist() == [1, 2, 2]             # unit plane: bits 0, 65, 129
    assert Pl[1, 0].tolist() == [0, 2, 0]             # sign plane: element 65 is -1
