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
* ``freivalds`` / ``matmul_rows``: checks for sizes too large for the full
  product (a randomized identity test and exact sampled rows).
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


def _gf4_matvec(M: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = M x over GF(4) via the Section 4.3 decomposition on F_2 mat-vecs."""
    M0, M1 = (M & 1).astype(np.int64), ((M >> 1) & 1).astype(np.int64)
    x0, x1 = (x & 1).astype(np.int64), ((x >> 1) & 1).astype(np.int64)
    p00 = (M0 @ x0) & 1
    p11 = (M1 @ x1) & 1
    pss = ((M0 ^ M1) @ (x0 ^ x1)) & 1
    return ((p00 ^ p11) | ((pss ^ p00) << 1)).astype(np.int64)


def _ext_matvec(q: int, M: np.ndarray, x: np.ndarray, table: np.ndarray) -> np.ndarray:
    """y = M x over an extension field: products from the element table, summed
    coefficient by coefficient mod p."""
    p, n, _ = EXTENSIONS[q]
    prods = table[np.asarray(M, dtype=np.int64), np.asarray(x, dtype=np.int64)[None, :]].astype(np.int64)
    return sum((((prods // p ** j) % p).sum(axis=1) % p) * p ** j for j in range(n))


def _matvec_mod(q: int, M: np.ndarray, x: np.ndarray, rows_per_chunk: int = 2048, table=None) -> np.ndarray:
    """M x over F_q (GF(4), extension fields), row chunk by row chunk to bound memory."""
    out = np.empty(M.shape[0], dtype=np.int64)
    for r in range(0, M.shape[0], rows_per_chunk):
        blk = M[r:r + rows_per_chunk]
        if q == 4:
            out[r:r + rows_per_chunk] = _gf4_matvec(blk, x)
        elif q in EXTENSIONS:
            out[r:r + rows_per_chunk] = _ext_matvec(q, blk, x, table)
        else:
            out[r:r + rows_per_chunk] = (blk.astype(np.int64) @ x) % q
    return out


def freivalds(q: int, A: np.ndarray, B: np.ndarray, C: np.ndarray, trials: int = 32,
              seed: int = 0) -> bool:
    """Randomized check that C = A B: for random x, A (B x) == C x over F_q.

    A wrong C passes one trial with probability at most 1/q (Freivalds), so the
    false-pass probability is at most q^-trials.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    A = np.asarray(A)
    B = np.asarray(B)
    C = np.asarray(C)
    n = B.shape[1]
    table = ext_mul_table(q) if q in EXTENSIONS and q != 4 else None
    for _ in range(trials):
        x = rng.integers(0, q, size=n, dtype=np.int64)
        lhs = _matvec_mod(q, A, _matvec_mod(q, B, x, table=table), table=table)
        rhs = _matvec_mod(q, C, x, table=table)
        if not np.array_equal(lhs, rhs):
            return False
    return True
