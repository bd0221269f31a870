"""The Four-Russians kernels' accumulation formulas, restated bit by bit and
checked exhaustively against integer arithmetic (no GPU).

The device code (csrc/fq_fields.cuh) accumulates the D = 3 lookups of a k-row
block, acc += t0 + 2 t1 + 4 t2, with carry-save adders instead of three field
additions (Section 4.2's add): F_7 works mod 7 (8 = 1, so a carry out of bit
2 wraps to bit 0), F_5 mod 15 = 3 * 5 in four bits (16 = 1), folding to a
three-bit F_5 code with Section 4.2's fold5 only when the product is stored.
Here every formula is run on single bits for every input, and the result must
equal the integer sum modulo 7 or 15."""
import itertools

import pytest


def bits(x, n):
    return [(x >> i) & 1 for i in range(n)]


def value(b):
    return sum(v << i for i, v in enumerate(b))


def xor3(a, b, c):
    return a ^ b ^ c


def maj(a, b, c):
    return (a & b) | (a & c) | (b & c)


# ------------------------------------------------------------------- F_7 --

def f7_add(x, y):
    """Section 4.2's add with the carry out of bit 2 added back at bit 0."""
    s0, c0 = x[0] ^ y[0], x[0] & y[0]
    s1, c1 = xor3(x[1], y[1], c0), maj(x[1], y[1], c0)
    s2, s3 = xor3(x[2], y[2], c1), maj(x[2], y[2], c1)
    d0 = s0 & s3
    return [s0 ^ s3, s1 ^ d0, s2 ^ (s1 & d0)]


def f7_csa(x, y, z):
    s = [xor3(x[i], y[i], z[i]) for i in range(3)]
    m = [maj(x[i], y[i], z[i]) for i in range(3)]
    return s, [m[2], m[0], m[1]]          # the carry out of bit 2 has weight 8 = 1 mod 7


def f7_accumulate(acc, t0, t1, t2):
    d1 = [t1[2], t1[0], t1[1]]            # 2 t1: a rotation mod 7
    d2 = [t2[1], t2[2], t2[0]]            # 4 t2
    s1, c1 = f7_csa(t0, d1, d2)
    s2, c2 = f7_csa(acc, s1, c1)
    return f7_add(s2, c2)


def test_f7_accumulate_every_input():
    for acc, t0, t1, t2 in itertools.product(range(8), repeat=4):
        got = value(f7_accumulate(bits(acc, 3), bits(t0, 3), bits(t1, 3), bits(t2, 3)))
        assert got % 7 == (acc + t0 + 2 * t1 + 4 * t2) % 7, (acc, t0, t1, t2)


# ------------------------------------------------------------------- F_5 --

def fold5(s0, s1, s2, s3):
    """Section 4.2's eight-operation fold5: four bits to three, same value mod 5."""
    t = s2 | s1
    r2 = s0 ^ t
    r1 = (r2 & s0) ^ (s3 ^ s1)
    r0 = (t ^ s2) | (r1 & s3)
    return [r0, r1, r2]


def f5_accumulate15(acc, t0, t1, t2):
    """acc (four bits, mod 15) += t0 + 2 t1 + 4 t2 for three-bit codes t_d:
    a carry-save adder on t0, 2 t1 = (0, t1_0, t1_1, t1_2) and 4 t2 = (t2_2,
    0, t2_0, t2_1), one with acc, then a four-bit add whose carry out is
    added back at bit 0 -- no fold."""
    s = [t0[0] ^ t2[2], t0[1] ^ t1[0], xor3(t0[2], t1[1], t2[0]), t1[2] ^ t2[1]]
    m = [t0[0] & t2[2], t0[1] & t1[0], maj(t0[2], t1[1], t2[0]), t1[2] & t2[1]]
    c = [m[3], m[0], m[1], m[2]]
    u = [xor3(acc[i], s[i], c[i]) for i in range(4)]
    v = [maj(acc[i], s[i], c[i]) for i in range(4)]
    w = [v[3], v[0], v[1], v[2]]
    r = [u[0] ^ w[0]]
    k = u[0] & w[0]
    for i in range(1, 4):
        r.append(xor3(u[i], w[i], k))
        k = maj(u[i], w[i], k)
    a0 = r[0] & k
    b0 = r[1] & a0
    return [r[0] ^ k, r[1] ^ a0, r[2] ^ b0, r[3] ^ (r[2] & b0)]


def test_f5_accumulate_mod15_every_input():
    for acc, t0, t1, t2 in itertools.product(range(16), range(8), range(8), range(8)):
        got = value(f5_accumulate15(bits(acc, 4), bits(t0, 3), bits(t1, 3), bits(t2, 3)))
        assert 0 <= got <= 15
        assert got % 15 == (acc + t0 + 2 * t1 + 4 * t2) % 15, (acc, t0, t1, t2)


@pytest.mark.parametrize("acc", range(16))
def test_f5_fold_of_the_mod15_accumulator(acc):
    """The stored code: fold5 of the four-bit accumulator has its value mod 5."""
    assert value(fold5(*bits(acc, 4))) % 5 == acc % 5
