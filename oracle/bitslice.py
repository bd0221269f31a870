"""TEST INFRASTRUCTURE ONLY -- the paper's bitsliced element arithmetic, written out.

Every function takes and returns bit-planes (numpy ``uint64`` arrays, or any
objects with ``& | ^ ~``): bit position b of plane i holds bit i of the code of
element b, so one call operates on 64 elements per word (Section 3).

The formulas follow Sections 3 and 4 of Boothby & Bradshaw in their notation.
Four printed formulas are wrong as printed; each is given here twice, once as
printed (suffix ``_printed``, kept so the tests can show that it fails) and once
in the reading used everywhere else:

* F_3 add (Section 4.1): the printed r_0 and r_1 are swapped.
* F_7 reduce (Section 4.2): the common term must be a0 AND a1 AND a2, not OR.
* fold5, 13-operation form (Section 4.2): the outputs r_0, r_1 need OR with e_3.
* F_5 reduce (Section 4.2): no single-operator or wiring change repairs it; the
  canonical reduction is replaced by a derived one (``f5_reduce``).

Nothing here is shared with the CUDA path.
"""
from __future__ import annotations


# ---------------------------------------------------------------- Section 3 --

def z4_add(a0, a1, b0, b1):
    """Z/4 add of bitsliced 2-bit numbers a1a0 + b1b0 (Section 3, four operations)."""
    r0 = a0 ^ b0
    r1 = (a1 ^ b1) ^ (a0 & b0)
    return r0, r1


# -------------------------------------------------------------- Section 4.1 --
# F_3 representation: 0 = (x0, x1) = (0, 0), 1 = (1, 0), -1 = (1, 1); x0 marks a
# unit, x1 its sign.  Additive basis {1, -1}.

def f3_add_printed(x0, x1, y0, y1):
    """F_3 add exactly as printed in Section 4.1 (wrong: outputs swapped)."""
    u = x0 ^ y1
    v = x1 ^ y0
    s = u ^ x1                      # x0 + y1 + x1
    t = v ^ y1                      # x1 + y0 + y1
    r0 = u & v
    r1 = s | t
    return r0, r1


def f3_add(x0, x1, y0, y1):
    """F_3 add, Section 4.1 with r_0 and r_1 exchanged (six operations)."""
    u = x0 ^ y1
    v = x1 ^ y0
    s = u ^ x1                      # x0 + y1 + x1
    t = v ^ y1                      # x1 + y0 + y1
    r0 = s | t
    r1 = u & v
    return r0, r1


def f3_neg(a0, a1):
    """F_3 negation, Section 4.1: (r0, r1) = (a0, a0 xor a1)."""
    return a0, a0 ^ a1


def f3_sub(x0, x1, y0, y1):
    """F_3 subtraction x - y, Section 4.1 as printed (six operations)."""
    t = x0 ^ y0
    r0 = t | (x1 ^ y1)
    r1 = (t ^ y1) & (y0 ^ x1)
    return r0, r1


# -------------------------------------------------------------- Section 4.2 --
# F_5 and F_7: plain binary codes a2a1a0 (value a0 + 2 a1 + 4 a2 read mod p),
# not unique; additive basis {1, 2, 4}.

def ripple_add(a, b):
    """Grade-school binary add of bit lists (least significant first), Section 4.2.

    With len(b) = m <= n = len(a) this uses m - 1 full adders and n - m + 1 half
    adders; the result has n + 1 bits (the last is the carry out).
    """
    if len(b) > len(a):
        a, b = b, a
    out = []
    carry = None
    for i, ai in enumerate(a):
        if i < len(b):
            if carry is None:                       # half adder on a_0 + b_0
                s, carry = ai ^ b[i], ai & b[i]
            else:                                   # full adder
                u = ai ^ b[i]
                s = u ^ carry
                carry = (ai & b[i]) | (u & carry)
        else:                                       # half adder: bit + carry
            s, carry = ai ^ carry, ai & carry
        out.append(s)
    out.append(carry)
    return out


def f7_add(a, b):
    """F_7 add: s = add(a, b) (4 bits), r = add(s2s1s0, s3) (3 bits), Section 4.2."""
    s = ripple_add(list(a), list(b))
    r = ripple_add(s[:3], [s[3]])
    return tuple(r[:3])                              # r[3] is always 0


def f7_double(a):
    """F_7 double: a rotation of the three planes, Section 4.2."""
    a0, a1, a2 = a
    return a2, a0, a1


def f7_neg(a):
    """F_7 negation: complement every plane, Section 4.2."""
    a0, a1, a2 = a
    return ~a0, ~a1, ~a2


def f7_reduce_printed(a):
    """F_7 reduce as printed (wrong: OR where AND is needed)."""
    a0, a1, a2 = a
    o = a0 | a1 | a2
    return a0 ^ o, a1 ^ o, a2 ^ o


def f7_reduce(a):
    """F_7 canonical reduce, Section 4.2 with AND: maps code 7 to 0, others fixed."""
    a0, a1, a2 = a
    c = a0 & a1 & a2
    return a0 ^ c, a1 ^ c, a2 ^ c


def fold5_13_printed(s):
    """fold5 in the 13-operation form as printed (wrong: AND where OR is needed)."""
    s0, s1, s2, s3 = s
    n0, n1, n2 = ~s2, s3, ~s3
    e = ripple_add([n0, n1, n2], [s0, s1])
    return e[0] & e[3], e[1] & e[3], e[2]


def fold5_13(s):
    """fold5, 13-operation form of Section 4.2 read with OR on e_3."""
    s0, s1, s2, s3 = s
    n0, n1, n2 = ~s2, s3, ~s3
    e = ripple_add([n0, n1, n2], [s0, s1])
    return e[0] | e[3], e[1] | e[3], e[2]


def fold5(s):
    """fold5, the 8-operation form of Section 4.2 as printed.

    Folds the 4-bit s3s2s1s0 into 3 bits with the same value mod 5.
    """
    s0, s1, s2, s3 = s
    t = s2 | s1
    r2 = s0 ^ t
    r1 = (r2 & s0) ^ (s3 ^ s1)
    r0 = (t ^ s2) | (r1 & s3)
    return r0, r1, r2


def f5_add(a, b):
    """F_5 add: s = add(a, b), r = fold5(s), Section 4.2."""
    s = ripple_add(list(a), list(b))
    return fold5(tuple(s))


def f5_double(a):
    """F_5 double: fold5(a2 a1 a0 0), Section 4.2."""
    a0, a1, a2 = a
    zero = a0 ^ a0
    return fold5((zero, a0, a1, a2))


def f5_neg(a):
    """F_5 negation: fold5(a1 a0 0 a2), i.e. 4a = -a, Section 4.2."""
    a0, a1, a2 = a
    zero = a0 ^ a0
    return fold5((a2, zero, a0, a1))


def f5_reduce_printed(a):
    """F_5 reduce as printed in Section 4.2 (garbled: not a canonical reduction)."""
    a0, a1, a2 = a
    t = a0 ^ a1
    u = (a0 & a1) | t
    return u, (u | a2) ^ a0, u ^ t


def f5_reduce(a):
    """F_5 canonical reduce (derived; replaces the garbled printed one).

    Codes 5, 6, 7 become 0, 1, 2; codes 0..4 are unchanged.
    c = a2 and (a0 or a1) marks codes 5..7.
    """
    a0, a1, a2 = a
    c = a2 & (a0 | a1)
    r0 = (a0 & ~c) | (c & a1 & ~a0)
    r1 = a1 & (~c | a0)
    r2 = a2 & ~c
    return r0, r1, r2


# -------------------------------------------------------------- Section 4.3 --
# GF(4) = F_2[x]/(x^2 + x + 1), element a0 + alpha a1: two planes, add is XOR.

def gf4_add(x0, x1, y0, y1):
    return x0 ^ y0, x1 ^ y1


def gf4_mul_alpha(a0, a1):
    """alpha * (a0 + alpha a1) = a1 + alpha (a0 + a1), using alpha^2 = alpha + 1."""
    return a1, a0 ^ a1
