"""TEST INFRASTRUCTURE ONLY -- the paper's Four-Russians product, step by step.

A slow, literal rendering of Section 2 over the bitsliced rows of Sections 3-4,
for small matrices.  It exists to pin the reading of the method (the additive
basis, the maps phi_d, the binary-combination tables and the scaling by
alpha_d) against the plain product in ``oracle.matmul``:

    C_i = sum_s sum_d alpha_d * T_s[ phi_d(a_{i,sk}), ..., phi_d(a_{i,sk+k-1}) ]

where T_s[b] = sum_{t<k} b_t B_{sk+t} is the table of binary combinations of the
k rows of block s (Section 2; the sum indices printed as t = 0..t-1 mean
t = 0..k-1).  When k does not divide l the last block has fewer rows, which is
the same as padding A with zero columns and B with zero rows.

Element arithmetic is the formulas of ``oracle.bitslice``; rows are arrays of
shape (planes, words).
"""
from __future__ import annotations

import numpy as np

from . import bitslice as bs
from . import encoding


class _Field:
    """Bitsliced row arithmetic and additive basis for one field (Section 4)."""

    def __init__(self, q: int):
        self.q = q
        self.P = encoding.planes(q)

    # additive basis {alpha_d} and the maps phi_d : K -> {0, 1} (Section 2)
    def basis_size(self) -> int:
        return {2: 1, 3: 2, 4: 2, 5: 3, 7: 3}[self.q]

    def phi(self, d: int, values: np.ndarray) -> np.ndarray:
        v = np.asarray(values).astype(np.int64)
        if self.q == 3:        # basis {1, -1}: a = phi_0(a) - phi_1(a)
            return (v == 1).astype(np.int64) if d == 0 else (v == 2).astype(np.int64)
        return (v >> d) & 1    # {1, 2, 4} for F_5, F_7; {1, alpha} for GF(4); {1} for F_2

    def add(self, x, y):
        q = self.q
        if q == 2:
            return (x[0] ^ y[0],)
        if q == 3:
            return bs.f3_add(x[0], x[1], y[0], y[1])
        if q == 4:
            return bs.gf4_add(x[0], x[1], y[0], y[1])
        if q == 5:
            return bs.f5_add(x, y)
        return bs.f7_add(x, y)

    def scale_by_basis(self, d: int, x):
        """alpha_d * x for the basis element alpha_d."""
        q = self.q
        if d == 0:
            return x
        if q == 3:             # alpha_1 = -1
            return bs.f3_neg(x[0], x[1])
        if q == 4:             # alpha_1 = alpha
            return bs.gf4_mul_alpha(x[0], x[1])
        r = x                  # alpha_d = 2^d, Horner-free: double d times
        for _ in range(d):
            r = bs.f5_double(r) if q == 5 else bs.f7_double(r)
        return r


def m4rm(q: int, A: np.ndarray, B: np.ndarray, k: int) -> np.ndarray:
    """C = A B over F_q by the method of Section 2; returns residues (m, n)."""
    A = np.asarray(A)
    B = np.asarray(B)
    m, l = A.shape
    l2, n = B.shape
    if l != l2 or k < 1:
        raise ValueError("shape mismatch or bad k")
    F = _Field(q)
    Bp = encoding.pack(q, B)                      # (P, l, W)
    W = Bp.shape[2]
    zero = tuple(np.zeros(W, dtype=np.uint64) for _ in range(F.P))
    C = [zero for _ in range(m)]
    nblocks = (l + k - 1) // k
    for s in range(nblocks):
        rows = list(range(s * k, min(l, s * k + k)))
        # T_s[b] for every b in {0,1}^k: T[b] = T[b without its lowest set bit] + B_row
        T = [zero] * (1 << k)
        for b in range(1, 1 << k):
            t = (b & -b).bit_length() - 1
            Brow = tuple(Bp[p, rows[t]] for p in range(F.P)) if t < len(rows) else zero
            T[b] = F.add(T[b & (b - 1)], Brow)
        for i in range(m):
            for d in range(F.basis_size()):
                bits = F.phi(d, A[i, rows])
                idx = int(sum(int(bit) << t for t, bit in enumerate(bits)))
                C[i] = F.add(C[i], F.scale_by_basis(d, T[idx]))
    Cp = np.stack([np.stack([C[i][p] for i in range(m)]) for p in range(F.P)]) if m else \
        np.zeros((F.P, 0, W), dtype=np.uint64)
    return encoding.unpack(q, Cp, n)
