"""TEST INFRASTRUCTURE ONLY -- the bitsliced representation of residue matrices.

Section 3 stores bit i of every element's code in plane i; Section 4 fixes the
codes:

* F_3 (Section 4.1): 0 -> (x0, x1) = (0, 0), 1 -> (1, 0), -1 = 2 -> (1, 1).
* F_5, F_7 (Section 4.2): the binary digits of the residue, (a0, a1, a2);
  any 3-bit code is accepted on decode and read mod p (codes are not unique).
* GF(4) (Section 4.3): element a0 + alpha a1 has code a0 + 2 a1, planes (a0, a1).
* F_2: one plane.
* F_{p^n} (``fields.EXTENSIONS``; Section 4.3's matrix-level view A = sum_j A_j
  x^j): code sum_j c_j p^j; the planes of coefficient matrix A_0 (F_p codes
  above), then those of A_1, and so on.  GF(4) is the case p = 2, n = 2.

Word layout (a choice of this library; the paper's display puts element 0 at the
left): element j of a row is bit (j mod 64) of 64-bit word floor(j / 64).
``pack`` returns an array of shape (planes, rows, ceil(cols / 64)).
"""
from __future__ import annotations

import numpy as np

from .fields import EXTENSIONS

PLANES = {2: 1, 3: 2, 4: 2, 5: 3, 7: 3}


def planes(q: int) -> int:
    if q in EXTENSIONS:
        p, n, _ = EXTENSIONS[q]
        return n * PLANES[p]
    if q not in PLANES:
        raise ValueError("unsupported field size %r" % (q,))
    return PLANES[q]


def codes_to_bits(q: int, values: np.ndarray) -> list[np.ndarray]:
    """Per-element code bits (list over planes of 0/1 uint8 arrays)."""
    v = np.asarray(values).astype(np.uint8)
    if np.any(v >= q):
        raise ValueError("residue out of range for q=%d" % q)
    if q in EXTENSIONS and q != 4:
        p, n, _ = EXTENSIONS[q]
        out = []
        for j in range(n):
            out += codes_to_bits(p, (v.astype(np.int64) // p ** j) % p)
        return out
    if q == 3:
        unit = (v != 0).astype(np.uint8)
        sign = (v == 2).astype(np.uint8)
        return [unit, sign]
    return [((v >> i) & 1).astype(np.uint8) for i in range(planes(q))]


def bits_to_values(q: int, bits: list[np.ndarray]) -> np.ndarray:
    """Decode per-element code bits to residues in [0, q)."""
    b = [np.asarray(x).astype(np.int64) for x in bits]
    if q in EXTENSIONS and q != 4:
        p, n, _ = EXTENSIONS[q]
        P = PLANES[p]
        return sum(bits_to_values(p, b[j * P:(j + 1) * P]).astype(np.int64) * p ** j
                   for j in range(n)).astype(np.uint8)
    if q == 3:
        x0, x1 = b
        if np.any((x0 == 0) & (x1 == 1)):
            raise ValueError("F_3 code (0, 1) is not a valid element")
        return np.where(x0 == 0, 0, np.where(x1 == 0, 1, 2)).astype(np.uint8)
    val = sum(bi << i for i, bi in enumerate(b))
    if q == 4:
        return val.astype(np.uint8)
    return (val % q).astype(np.uint8)


def _bits_to_words(bits: np.ndarray) -> np.ndarray:
    """(rows, cols) 0/1 -> (rows, ceil(cols/64)) uint64, element j at bit j % 64."""
    rows, cols = bits.shape
    words = (cols + 63) // 64
    padded = np.zeros((rows, words * 64), dtype=np.uint64)
    padded[:, :cols] = bits
    shifts = np.arange(64, dtype=np.uint64)
    return (padded.reshape(rows, words, 64) << shifts).sum(axis=2, dtype=np.uint64)


def _words_to_bits(words: np.ndarray, cols: int) -> np.ndarray:
    rows, nw = words.shape
    shifts = np.arange(64, dtype=np.uint64)
    bits = (words[:, :, None] >> shifts) & np.uint64(1)
    return bits.reshape(rows, nw * 64)[:, :cols].astype(np.uint8)


def pack(q: int, R: np.ndarray) -> np.ndarray:
    """Residue matrix -> bit-planes, shape (planes, rows, ceil(cols / 64))."""
    R = np.asarray(R)
    if R.ndim != 2:
        raise ValueError("expected a matrix")
    return np.stack([_bits_to_words(b) for b in codes_to_bits(q, R)])


def unpack(q: int, planes_arr: np.ndarray, cols: int) -> np.ndarray:
    """Bit-planes (planes, rows, words) -> residue matrix (rows, cols)."""
    P = planes(q)
    if planes_arr.shape[0] != P:
        raise ValueError("expected %d planes" % P)
    return bits_to_values(q, [_words_to_bits(planes_arr[i], cols) for i in range(P)])
