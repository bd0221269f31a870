"""TEST INFRASTRUCTURE ONLY -- the CPU oracle for matrix products over small fields.

Boothby & Bradshaw, "Bitslicing and the Method of Four Russians Over Larger
Finite Fields".  This package is the plain, slow, obviously correct statement of
what the library computes; the CUDA path is checked against it bit for bit.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import it.  It imports nothing from the library and the
library imports nothing from it.

* ``matmul(q, A, B)``: C = AB over F_q (q = 2, 3, 5, 7), GF(4) (q = 4) or an
  extension field F_{p^n} (q = 8, 9, 25, 27, 49, 125; ``fields.EXTENSIONS``), on
  code matrices (uint8, entries in [0, q)), computed in C as the row
  combination C_i = sum_j a_ij B_j of Section 2 (``fq_oracle.c``).
* ``gf4_karatsuba(A, B)``: the matrix-level GF(4) formula of Section 4.3 over
  three F_2 products, a second GF(4) oracle.
* ``ext_karatsuba(q, A, B)``: the matrix-level products of Section 4.3 for any
  extension field (Karatsuba for degree 2, the paper's six-product trinomial
  formula for degree 3) over base-field products, then reduction by the
  defining polynomial: a second oracle for the extension fields.
* ``encoding``: the bitsliced representation (Sections 3-4).
* ``bitslice``: the paper's element formulas.
* ``m4rm``: the Section 2 method itself, step by step, for small sizes.
* ``freivalds`` / ``matmul_rows`` / ``matmul_cols``: checks for sizes too
  large for the full product (a randomized identity test, exact sampled rows
  and exact sampled columns).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import bitslice, encoding, fields  # noqa: F401
from .build import build as _build
from .fields import EXTENSIONS

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build()
        lib = ctypes.CDLL(path)
        i64 = ctypes.c_int64
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.fq_oracle_matmul_fp.argtypes = [ctypes.c_int, i64, i64, i64, u8p, i64, u8p, i64, u8p, i64,
                                            ctypes.c_int]
        lib.fq_oracle_matmul_fp.restype = ctypes.c_int
        lib.fq_oracle_matmul_gf4.argtypes = [i64, i64, i64, u8p, i64, u8p, i64, u8p, i64, ctypes.c_int]
        lib.fq_oracle_matmul_gf4.restype = ctypes.c_int
        lib.fq_oracle_matmul_ext.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64, i64,
                                             i64, u8p, i64, u8p, i64, u8p, i64, ctypes.c_int]
        lib.fq_oracle_matmul_ext.restype = ctypes.c_int
        lib.fq_oracle_threads.argtypes = [ctypes.c_int]
        lib.fq_oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


FIELDS = fields.FIELDS


def threads_used(threads: int = 0) -> int:
    """Number of host threads ``matmul`` uses for a given request (0 = all)."""
    return int(_load().fq_oracle_threads(int(threads)))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def matmul(q: int, A: np.ndarray, B: np.ndarray, threads: int = 0) -> np.ndarray:
    """C = A B over F_q (q prime <= 7, GF(4) or an extension field); codes in, codes out."""
    if q not in FIELDS:
        raise ValueError("unsupported field size %r" % (q,))
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[0]:
        raise ValueError("shape mismatch")
    if A.size and A.max() >= q or B.size and B.max() >= q:
        raise ValueError("residue out of range")
    m, l = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), dtype=np.uint8)
    lib = _load()
    if q == 4:
        rc = lib.fq_oracle_matmul_gf4(m, l, n, _ptr(A), l, _ptr(B), n, _ptr(C), n, int(threads))
    elif q in EXTENSIONS:
        return matmul_ext(q, A, B, threads)
    else:
        rc = lib.fq_oracle_matmul_fp(q, m, l, n, _ptr(A), l, _ptr(B), n, _ptr(C), n, int(threads))
    if rc != 0:
        raise RuntimeError("oracle failed with status %d" % rc)
    return C


def matmul_ext(q: int, A: np.ndarray, B: np.ndarray, threads: int = 0) -> np.ndarray:
    """C = A B over the extension field q of ``fields.EXTENSIONS`` (GF(4) included)
    by the tabulated element arithmetic of ``fq_oracle_matmul_ext``."""
    p, n, r = EXTENSIONS[q]
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[0]:
        raise ValueError("shape mismatch")
    m, l = A.shape
    nn = B.shape[1]
    C = np.zeros((m, nn), dtype=np.uint8)
    rr = (ctypes.c_int * n)(*r)
    rc = _load().fq_oracle_matmul_ext(p, n, rr, m, l, nn, _ptr(A), l, _ptr(B), nn, _ptr(C), nn, int(threads))
    if rc != 0:
        raise RuntimeError("oracle failed with status %d" % rc)
    return C


def digits(q: int, X: np.ndarray) -> list[np.ndarray]:
    """Coefficient matrices X_0 .. X_{n-1} over F_p of X = sum_j X_j x^j."""
    p, n, _ = EXTENSIONS[q]
    X = np.asarray(X).astype(np.int64)
    return [((X // p ** j) % p).astype(np.uint8) for j in range(n)]


def compose(q: int, ds) -> np.ndarray:
    """Inverse of ``digits``."""
    p, n, _ = EXTENSIONS[q]
    return sum(np.asarray(d).astype(np.int64) * p ** j for j, d in enumerate(ds)).astype(np.uint8)


def ext_karatsuba(q: int, A: np.ndarray, B: np.ndarray, threads: int = 0) -> np.ndarray:
    """Product over an extension field by Section 4.3's matrix-level method:
    A = sum_j A_j x^j, B = sum_j B_j x^j with A_j, B_j over F_p; the polynomial
    product's coefficients c_k from Karatsuba (degree 2: three products) or the
    paper's six-product trinomial formula (degree 3), each a base-field matrix;
    then x^k (k >= n) is replaced using the defining polynomial."""
    p, n, r = EXTENSIONS[q]
    a, b = digits(q, A), digits(q, B)
    mm = lambda X, Y: matmul(p, X, Y, threads).astype(np.int64)
    plus = lambda X, Y: (np.asarray(X).astype(np.int64) + Y) % p
    if n == 2:
        p00, p11 = mm(a[0], b[0]), mm(a[1], b[1])
        pss = mm(plus(a[0], a[1]), plus(b[0], b[1]))
        c = [p00, pss - p00 - p11, p11]
    elif n == 3:
        a0b0, a1b1, a2b2 = mm(a[0], b[0]), mm(a[1], b[1]), mm(a[2], b[2])
        c = [a0b0,
             mm(plus(a[0], a[1]), plus(b[0], b[1])) - a0b0 - a1b1,
             mm(plus(a[0], a[2]), plus(b[0], b[2])) - a0b0 - a2b2 + a1b1,
             mm(plus(a[2], a[1]), plus(b[2], b[1])) - a2b2 - a1b1,
             a2b2]
    else:
        raise ValueError("degree %d" % n)
    for k in range(2 * n - 2, n - 1, -1):          # x^k = x^(k-n) (r_0 + r_1 x + ...)
        for j in range(n):
            c[k - n + j] = c[k - n + j] + r[j] * c[k]
        c[k] = 0
    return compose(q, [np.mod(c[j], p) for j in range(n)])


def ext_mul_table(q: int) -> np.ndarray:
    """q x q table of element products, from the oracle's own 1 x 1 products
    (an outer product of the column 0..q-1 with the row 0..q-1)."""
    e = np.arange(q, dtype=np.uint8)
    return matmul(q, e.reshape(q, 1), e.reshape(1, q))


def matmul_rows(q: int, A: np.ndarray, B: np.ndarray, rows, threads: int = 0) -> np.ndarray:
    """Exact rows ``rows`` of A B (each row is C_i = A_i B, independent of the rest)."""
    rows = np.asarray(rows, dtype=np.int64)
    return matmul(q, np.asarray(A)[rows], B, threads)


def matmul_cols(q: int, A: np.ndarray, B: np.ndarray, cols, threads: int = 0) -> np.ndarray:
    """Exact columns ``cols`` of A B, as a len(A) x len(cols) matrix: column j of
    the product is A times column j of B, independent of the other columns."""
    cols = np.asarray(cols, dtype=np.int64)
    return matmul(q, A, np.ascontiguousarray(np.asarray(B)[:, cols]), threads)


def gf4_karatsuba(A: np.ndarray, B: np.ndarray, threads: int = 0) -> np.ndarray:
    """GF(4) product by Section 4.3: with A = A0 + alpha A1 and B = B0 + alpha B1,
    AB = (A0 B0 + A1 B1) + alpha ((A0 + A1)(B0 + B1) + A0 B0), three F_2 products."""
    A = np.asarray(A, dtype=np.uint8)
    B = np.asarray(B, dtype=np.uint8)
    A0, A1 = A & 1, (A >> 1) & 1
    B0, B1 = B & 1, (B >> 1) & 1
    P00 = matmul(2, A0, B0, threads)
    P11 = matmul(2, A1, B1, threads)
    Pss = matmul(2, A0 ^ A1, B0 ^ B1, threads)
    c0 = P00 ^ P11
    c1 = Pss ^ P00
    return (c0 | (c1 << 1)).astype(np.uint8)


# Largest integer below which every float64 value is exact: the library
# matmul below only ever adds non-negative integers, so while the longest sum
# stays under this bound no rounding can happen, whatever the summation order.
_FLOAT64_EXACT = 2 ** 53


def _fp_matmul(p: int, M: np.ndarray, X: np.ndarray, chunk_bytes: int = 1 << 28) -> np.ndarray:
    """(M X) mod p for M with entries in [0, p) (uint8) and X with entries in
    [0, p) (int64), by a float64 library matmul over row chunks of M.  Each
    entry of M X is a sum of cols(M) products of at most (p - 1)^2, so it is an
    exact float64 integer while cols(M) (p - 1)^2 < 2^53."""
    M = np.asarray(M)
    r, c = M.shape
    if c * (p - 1) ** 2 >= _FLOAT64_EXACT:
        raise ValueError("sums of %d terms could exceed 2^53" % c)
    Xf = np.asarray(X, dtype=np.float64)
    out = np.empty((r, Xf.shape[1]), dtype=np.int64)
    step = max(1, chunk_bytes // max(1, 8 * c))
    for i in range(0, r, step):
        out[i:i + step] = np.mod(M[i:i + step].astype(np.float64) @ Xf, p).astype(np.int64)
    return out


def _field_matmul(q: int, M: np.ndarray, X: np.ndarray, chunk_bytes: int = 1 << 28) -> np.ndarray:
    """M X over F_q on codes (M uint8, X int64), for the randomized check.

    F_p: ``_fp_matmul``.  F_{p^n} (GF(4) included): with M = sum_a M_a x^a and
    X = sum_b X_b x^b over F_p (the code digits), the polynomial product's
    coefficient k is sum_{a + b = k} M_a X_b (schoolbook, n^2 base-field
    products), and x^k for k >= n is replaced, highest first, using the defining
    polynomial x^n = r_0 + r_1 x + ... (Section 4.3's extension fields)."""
    if q not in EXTENSIONS:
        return _fp_matmul(q, M, X, chunk_bytes)
    p, n, r = EXTENSIONS[q]
    M = np.asarray(M, dtype=np.uint8)
    ms = [(M // p ** j) % p for j in range(n)]
    xs = [((np.asarray(X, dtype=np.int64) // p ** j) % p) for j in range(n)]
    c = [0] * (2 * n - 1)
    for a in range(n):
        for b in range(n):
            c[a + b] = c[a + b] + _fp_matmul(p, ms[a], xs[b], chunk_bytes)
    for k in range(2 * n - 2, n - 1, -1):
        for j in range(n):
            c[k - n + j] = c[k - n + j] + r[j] * c[k]
        c[k] = 0
    return sum(np.mod(c[j], p) * p ** j for j in range(n))


def freivalds(q: int, A: np.ndarray, B: np.ndarray, C: np.ndarray, trials: int = 32,
              seed: int = 0, chunk_bytes: int = 1 << 28) -> bool:
    """Randomized check that C = A B over F_q (Freivalds): for a random n x trials
    matrix X over F_q, A (B X) == C X.

    Each column of X is an independent uniform vector; if C != A B, one column
    passes with probability at most 1/q, so a wrong C passes with probability at
    most q^-trials.  All products are computed exactly (``_field_matmul``).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    A = np.asarray(A)
    B = np.asarray(B)
    C = np.asarray(C)
    if A.shape[1] != B.shape[0] or C.shape != (A.shape[0], B.shape[1]):
        raise ValueError("shape mismatch")
    X = rng.integers(0, q, size=(B.shape[1], trials), dtype=np.int64)
    lhs = _field_matmul(q, A, _field_matmul(q, B, X, chunk_bytes), chunk_bytes)
    rhs = _field_matmul(q, C, X, chunk_bytes)
    return bool(np.array_equal(lhs, rhs))
