"""The paper's bitsliced element formulas, checked exhaustively against integer
arithmetic mod q; the printed misprints are shown to fail."""
import itertools

import numpy as np
import pytest

from oracle import bitslice as bs

U = np.uint64


def planes_for(codes, nbits):
    """codes: list of ints, one per bit position -> list of nbits uint64 words."""
    assert len(codes) <= 64
    out = []
    for i in range(nbits):
        w = 0
        for pos, c in enumerate(codes):
            w |= ((c >> i) & 1) << pos
        out.append(U(w))
    return out


def codes_of(planes, count):
    return [sum(((int(p) >> pos) & 1) << i for i, p in enumerate(planes)) for pos in range(count)]


# F_3 codes as (x0, x1) -> value
F3_CODE = {0: 0b00, 1: 0b01, 2: 0b11}     # bit 0 = x0 (unit), bit 1 = x1 (sign)
F3_VAL = {v: k for k, v in F3_CODE.items()}


def f3_pairs():
    return list(itertools.product(range(3), repeat=2))


def _f3_apply(fn):
    pairs = f3_pairs()
    x = planes_for([F3_CODE[a] for a, _ in pairs], 2)
    y = planes_for([F3_CODE[b] for _, b in pairs], 2)
    r = fn(x[0], x[1], y[0], y[1])
    return pairs, codes_of(r, len(pairs))


def test_f3_add_reading_is_exact():
    pairs, out = _f3_apply(bs.f3_add)
    for (a, b), c in zip(pairs, out):
        assert c in F3_VAL, "add produced the unused code (0, 1)"
        assert F3_VAL[c] == (a + b) % 3


def test_f3_add_as_printed_fails():
    pairs, out = _f3_apply(bs.f3_add_printed)
    wrong = [(a, b) for (a, b), c in zip(pairs, out) if F3_VAL.get(c) != (a + b) % 3]
    assert (0, 1) in wrong          # 0 + 1 comes out as the unused code (0, 1)


def test_f3_sub_and_neg():
    pairs, out = _f3_apply(bs.f3_sub)
    for (a, b), c in zip(pairs, out):
        assert F3_VAL[c] == (a - b) % 3
    x = planes_for([F3_CODE[a] for a in range(3)], 2)
    r = bs.f3_neg(x[0], x[1])
    assert [F3_VAL[c] for c in codes_of(r, 3)] == [0, 2, 1]


def test_z4_add_section3():
    pairs = list(itertools.product(range(4), repeat=2))
    x = planes_for([a for a, _ in pairs], 2)
    y = planes_for([b for _, b in pairs], 2)
    r = bs.z4_add(x[0], x[1], y[0], y[1])
    assert codes_of(r, len(pairs)) == [(a + b) % 4 for a, b in pairs]


# ------------------------------------------------------------ F_5 and F_7 --

def _all_code_pairs(nbits):
    return list(itertools.product(range(1 << nbits), repeat=2))   # 64 pairs for 3 bits


@pytest.mark.parametrize("p,add", [(7, bs.f7_add), (5, bs.f5_add)])
def test_add_over_all_codes(p, add):
    pairs = _all_code_pairs(3)
    x = planes_for([a for a, _ in pairs], 3)
    y = planes_for([b for _, b in pairs], 3)
    out = codes_of(add(tuple(x), tuple(y)), len(pairs))
    for (a, b), c in zip(pairs, out):
        assert c < 8 and c % p == (a + b) % p


@pytest.mark.parametrize("p,fn,mult", [(7, bs.f7_double, 2), (7, bs.f7_neg, -1),
                                       (5, bs.f5_double, 2), (5, bs.f5_neg, -1)])
def test_unary_over_all_codes(p, fn, mult):
    x = planes_for(list(range(8)), 3)
    out = codes_of(fn(tuple(x)), 8)
    for a, c in enumerate(out):
        assert c % p == (mult * a) % p


@pytest.mark.parametrize("p,fn", [(7, bs.f7_reduce), (5, bs.f5_reduce)])
def test_reduce_is_canonical(p, fn):
    x = planes_for(list(range(8)), 3)
    out = codes_of(fn(tuple(x)), 8)
    assert out == [a % p for a in range(8)]


@pytest.mark.parametrize("p,fn", [(7, bs.f7_reduce_printed), (5, bs.f5_reduce_printed)])
def test_reduce_as_printed_fails(p, fn):
    x = planes_for(list(range(8)), 3)
    out = codes_of(fn(tuple(x)), 8)
    assert out != [a % p for a in range(8)]
    assert any(c % p != a % p for a, c in enumerate(out))   # not even value-preserving


def test_f7_reduce_printed_maps_one_to_six():
    x = planes_for([1], 3)
    assert codes_of(bs.f7_reduce_printed(tuple(x)), 1) == [6]


@pytest.mark.parametrize("fn", [bs.fold5, bs.fold5_13])
def test_fold5_preserves_value_mod5(fn):
    s = planes_for(list(range(16)), 4)
    out = codes_of(fn(tuple(s)), 16)
    for v, c in enumerate(out):
        assert c < 8 and c % 5 == v % 5


def test_fold5_13_outputs_in_2_to_7():
    s = planes_for(list(range(16)), 4)
    out = codes_of(bs.fold5_13(tuple(s)), 16)
    assert min(out) >= 2 and max(out) <= 7


def test_fold5_13_as_printed_fails():
    s = planes_for(list(range(16)), 4)
    out = codes_of(bs.fold5_13_printed(tuple(s)), 16)
    assert any(c % 5 != v % 5 for v, c in enumerate(out))


# ------------------------------------------------------------------ GF(4) --

GF4_MUL = {}
for a in range(4):
    GF4_MUL[(0, a)] = GF4_MUL[(a, 0)] = 0
    GF4_MUL[(1, a)] = GF4_MUL[(a, 1)] = a
GF4_MUL.update({(2, 2): 3, (2, 3): 1, (3, 2): 1, (3, 3): 2})   # x^2 = x + 1


def test_gf4_add_and_alpha():
    pairs = list(itertools.product(range(4), repeat=2))
    x = planes_for([a for a, _ in pairs], 2)
    y = planes_for([b for _, b in pairs], 2)
    assert codes_of(bs.gf4_add(x[0], x[1], y[0], y[1]), 16) == [a ^ b for a, b in pairs]
    z = planes_for(list(range(4)), 2)
    assert codes_of(bs.gf4_mul_alpha(z[0], z[1]), 4) == [GF4_MUL[(2, a)] for a in range(4)]


# ------------------------------------------- operation counts (Sections 3-4) --

class Op:
    """Counts the binary and unary bit operations a formula performs."""

    def __init__(self, counter):
        self.c = counter

    def _bin(self, other):
        self.c[0] += 1
        return Op(self.c)

    __and__ = __or__ = __xor__ = _bin

    def __invert__(self):
        self.c[0] += 1
        return Op(self.c)


def count_ops(fn, nargs, tuple_args=None):
    c = [0]
    if tuple_args is None:
        fn(*[Op(c) for _ in range(nargs)])
    else:
        fn(*[tuple(Op(c) for _ in range(k)) for k in tuple_args])
    return c[0]


def test_operation_counts():
    assert count_ops(bs.z4_add, 4) == 4               # Section 3: four operations
    assert count_ops(bs.f3_add, 4) == 6               # Section 4.1: six
    assert count_ops(bs.f3_sub, 4) == 6               # Section 4.1: six
    assert count_ops(bs.f3_neg, 2) == 1               # Section 4.1: one
    assert count_ops(bs.fold5, None, (4,)) == 8       # Section 4.2: eight
    assert count_ops(bs.f7_neg, None, (3,)) == 3      # Section 4.2: three
    assert count_ops(bs.f7_double, None, (3,)) == 0   # Section 4.2: zero
    assert count_ops(bs.f7_reduce, None, (3,)) == 5   # Section 4.2: five
    for m, n in ((1, 3), (2, 3), (3, 3), (2, 4)):     # add: 3m + 2n - 3 (m <= n)
        assert count_ops(lambda a, b: bs.ripple_add(list(a), list(b)), None, (n, m)) == 3 * m + 2 * n - 3
