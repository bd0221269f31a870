"""Pins for a matrix-product function over F_q: checks that fix the product by
something other than its own formula (library routines, closed forms, algebraic
identities, field axioms, the Frobenius automorphism, the defining polynomials
and the paper's matrix-level Karatsuba forms).  Each check takes ``mm(q, A, B)``
and returns True when the function passes."""
from __future__ import annotations

import numpy as np

from oracle.fields import EXTENSIONS


def rand(rng, q, r, c):
    return rng.integers(0, q, size=(r, c), dtype=np.int64).astype(np.uint8)


def gf4_add(X, Y):
    return (X ^ Y).astype(np.uint8)


def fadd(q, X, Y):
    if q == 4:
        return gf4_add(X, Y)
    if q in EXTENSIONS:                      # coefficientwise mod p
        p, n, _ = EXTENSIONS[q]
        X, Y = np.asarray(X).astype(np.int64), np.asarray(Y).astype(np.int64)
        return sum((((X // p ** j) + (Y // p ** j)) % p) * p ** j for j in range(n)).astype(np.uint8)
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


def mul_table(mm, q):
    """The q x q element products as 1 x 1 matrix products (one outer product)."""
    e = np.arange(q, dtype=np.uint8)
    return np.asarray(mm(q, e.reshape(q, 1), e.reshape(1, q))).astype(np.int64)


def check_field_axioms(mm, q, rng, samples=4000):
    """The element products of mm make F_q a field: 1 is the unit, 0 absorbs,
    products commute, every nonzero element has an inverse (so there are no
    zero divisors: the defining polynomial is irreducible), and products
    associate and distribute over coefficientwise addition (all triples for
    q <= 27, `samples` random triples above)."""
    T = mul_table(mm, q)
    e = np.arange(q)
    if not (np.array_equal(T[1], e) and not T[0].any() and np.array_equal(T, T.T)):
        return False
    if not all(1 in T[a, 1:] for a in range(1, q)):
        return False
    if q <= 27:
        a, b, c = (x.ravel() for x in np.meshgrid(e, e, e, indexing="ij"))
    else:
        a, b, c = (rng.integers(0, q, samples) for _ in range(3))
    if not np.array_equal(T[T[a, b], c], T[a, T[b, c]]):
        return False
    bc = fadd(q, b.astype(np.uint8), c.astype(np.uint8)).astype(np.int64)
    return np.array_equal(T[a, bc], fadd(q, T[a, b].astype(np.uint8), T[a, c].astype(np.uint8)))


def check_primitive(mm, q):
    """x (code p, the class of the polynomial variable) has multiplicative order
    q - 1: the defining polynomial is primitive, which singles it out among the
    irreducible ones a mistyped coefficient would give for most fields."""
    p, n, _ = EXTENSIONS[q]
    T = mul_table(mm, q)
    x, y = p, p
    for k in range(1, q):
        if y == 1:
            return k == q - 1
        y = int(T[y, x])
    return False


def check_frobenius(mm, q, rng):
    """The Frobenius map s(a) = a^p is a field automorphism, so applied to every
    entry it commutes with matrix products: s(AB) = s(A) s(B)."""
    p, n, _ = EXTENSIONS[q]
    T = mul_table(mm, q)
    frob = np.arange(q)
    for _ in range(p - 1):
        frob = T[frob, np.arange(q)]
    if len(set(frob.tolist())) != q or np.array_equal(frob, np.arange(q)):
        return False                          # a bijection other than the identity
    A, B = rand(rng, q, 9, 14), rand(rng, q, 14, 6)
    s = lambda X: frob[X.astype(np.int64)].astype(np.uint8)
    return np.array_equal(s(mm(q, A, B)), mm(q, s(A), s(B)))


def check_ext_karatsuba(mm, q, rng, karatsuba):
    """The product equals Section 4.3's matrix-level form over base-field products
    (Karatsuba for degree 2, the paper's trinomial formula for degree 3)."""
    for m, l, n in ((5, 9, 7), (33, 70, 40)):
        A, B = rand(rng, q, m, l), rand(rng, q, l, n)
        if not np.array_equal(mm(q, A, B), karatsuba(q, A, B)):
            return False
    return True


def run_all(mm, q, seed=0, karatsuba=None, ext_karatsuba=None):
    """All pins that apply to q; returns the names of the failing ones."""
    rng = np.random.default_rng(seed)
    fails = []
    checks = [("identity_perm", lambda: check_identity_perm(mm, q, rng)),
              ("units", lambda: check_units(mm, q)),
              ("identities", lambda: check_identities(mm, q, rng)),
              ("scalar", lambda: check_scalar(mm, q, rng))]
    if q in EXTENSIONS:
        checks.append(("field_axioms", lambda: check_field_axioms(mm, q, rng)))
        checks.append(("primitive", lambda: check_primitive(mm, q)))
        checks.append(("frobenius", lambda: check_frobenius(mm, q, rng)))
        if ext_karatsuba is not None:
            checks.append(("ext_karatsuba", lambda: check_ext_karatsuba(mm, q, rng, ext_karatsuba)))
    if q == 4:
        checks.append(("gf4_polynomial", lambda: check_gf4_polynomial(mm)))
        if karatsuba is not None:
            checks.append(("gf4_karatsuba", lambda: check_gf4_karatsuba(mm, rng, karatsuba)))
    elif q not in EXTENSIONS:
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
