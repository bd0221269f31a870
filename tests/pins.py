"""Pins for a matrix-product function over F_q: checks that fix the product by
something other than its own formula (library routines, closed forms, algebraic
identities, the GF(4) defining polynomial).  Each check takes ``mm(q, A, B)``
and returns True when the function passes."""
from __future__ import annotations

import numpy as np


def rand(rng, q, r, c):
    return rng.integers(0, q, size=(r, c), dtype=np.int64).astype(np.uint8)


def gf4_add(X, Y):
    return (X ^ Y).astype(np.uint8)


def fadd(q, X, Y):
    if q == 4:
        return gf4_add(X, Y)
    return ((X.astype(np.int64) + Y) % q).astype(np.uint8)


def check_numpy(mm, q, rng, shapes=((7, 13, 5), (64, 65, 63), (1, 200, 3), (33, 1, 17))):
    """F_p: agreement with numpy's int64 matmul reduced mod p."""
    assert q != 4
    for m, l, n in shapes:
        A, B = rand(rng, q, m, l), rand(rng, q, l, n)
        ref = (A.astype(np.int64) @ B.astype(np.int64)) % q
        if not np.array_equal(mm(q, A, B), ref.astype(np.uint8)):
            return False
    return True


def check_all_max(mm, q, lengths=(997, 1000, 1001, 4099)):
    """Closed form: A, B filled with p-1 give C = l (p-1)^2 mod p everywhere."""
    assert q != 4
    for l in lengths:
        A = np.full((3, l), q - 1, np.uint8)
        B = np.full((l, 4), q - 1, np.uint8)
        if not np.all(mm(q, A, B) == (l * (q - 1) ** 2) % q):
            return False
    return True


def check_identity_perm(mm, q, rng):
    """I B = B; a permutation matrix permutes rows; B I = B."""
    n = 11
    B = rand(rng, q, n, 9)
    I = np.eye(n, dtype=np.uint8)
    perm = rng.permutation(n)
    Pm = np.zeros((n, n), np.uint8)
    Pm[np.arange(n), perm] = 1
    if not np.array_equal(mm(q, I, B), B):
        return False
    if not np.array_equal(mm(q, Pm, B), B[perm]):
        return False
    return np.array_equal(mm(q, B, np.eye(9, dtype=np.uint8)), B)


def check_units(mm, q):
    """Matrix units: E_ij E_jk = E_ik and E_ij E_j'k = 0 for j != j' (3 x 4 x 5)."""
    for i in range(3):
        for j in range(4):
            for jj in range(4):
                for k in range(5):
                    A = np.zeros((3, 4), np.uint8)
                    A[i, j] = 1
                    B = np.zeros((4, 5), np.uint8)
                    B[jj, k] = 1
                    C = np.zeros((3, 5), np.uint8)
                    if j == jj:
                        C[i, k] = 1
                    if not np.array_equal(mm(q, A, B), C):
                        return False
    return True


def check_identities(mm, q, rng):
    """(AB)C = A(BC), A(B+B') = AB + AB', (AB)^T = B^T A^T on rectangular shapes."""
    A, B, B2, Cm = rand(rng, q, 9, 14), rand(rng, q, 14, 6), rand(rng, q, 14, 6), rand(rng, q, 6, 11)
    if not np.array_equal(mm(q, mm(q, A, B), Cm), mm(q, A, mm(q, B, Cm))):
        return False
    if not np.array_equal(mm(q, A, fadd(q, B, B2)), fadd(q, mm(q, A, B), mm(q, A, B2))):
        return False
    return np.array_equal(mm(q, A, B).T, mm(q, np.ascontiguousarray(B.T), np.ascontiguousarray(A.T)))


def check_scalar(mm, q, rng):
    """(cA)B = c(AB) for every scalar c, with c x computed as the 1x1 product."""
    A, B = rand(rng, q, 5, 8), rand(rng, q, 8, 7)
    AB = mm(q, A, B)
    for c in range(q):
        cm = np.array([[c]], np.uint8)
        cA = mm(q, A.reshape(-1, 1), cm).reshape(A.shape)
        cAB = mm(q, AB.reshape(-1, 1), cm).reshape(AB.shape)
        if not np.array_equal(mm(q, cA, B), cAB):
            return False
    return True


def check_gf4_polynomial(mm):
    """GF(4) = F_2[x]/(x^2 + x + 1) with codes c0 + 2 c1 <-> c0 + c1 x:
    x*x = x + 1, x*(x+1) = 1, (x+1)^2 = x, 1 is the unit, 0 absorbs."""
    table = {(2, 2): 3, (2, 3): 1, (3, 3): 2, (3, 2): 1}
    for a in range(4):
        table[(1, a)] = a
        table[(a, 1)] = a
        table[(0, a)] = 0
        table[(a, 0)] = 0
    for (a, b), c in table.items():
        if int(mm(4, np.array([[a]], np.uint8), np.array([[b]], np.uint8))[0, 0]) != c:
            return False
    return True


def check_gf4_karatsuba(mm, rng, karatsuba):
    """GF(4) product equals the Section 4.3 matrix-level formula over F_2."""
    for m, l, n in ((5, 9, 7), (40, 70, 33)):
        A, B = rand(rng, 4, m, l), rand(rng, 4, l, n)
        if not np.array_equal(mm(4, A, B), karatsuba(A, B)):
            return False
    return True


def run_all(mm, q, seed=0, karatsuba=None):
    """All pins that apply to q; returns the names of the failing ones."""
    rng = np.random.default_rng(seed)
    fails = []
    checks = [("identity_perm", lambda: check_identity_perm(mm, q, rng)),
              ("units", lambda: check_units(mm, q)),
              ("identities", lambda: check_identities(mm, q, rng)),
              ("scalar", lambda: check_scalar(mm, q, rng))]
    if q == 4:
        checks.append(("gf4_polynomial", lambda: check_gf4_polynomial(mm)))
        if karatsuba is not None:
            checks.append(("gf4_karatsuba", lambda: check_gf4_karatsuba(mm, rng, karatsuba)))
    else:
        checks.append(("numpy", lambda: check_numpy(mm, q, rng)))
        checks.append(("all_max", lambda: check_all_max(mm, q)))
    for name, fn in checks:
        try:
            ok = fn()
        except Exception:  # a mutant that breaks shapes fails the pin
            ok = False
        if not ok:
            fails.append(name)
    return fails
