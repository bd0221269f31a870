"""TEST INFRASTRUCTURE ONLY -- the fields the oracle knows.

Prime fields F_p (p = 2, 3, 5, 7) and extension fields F_{p^n} = F_p[x]/(f)
(Section 4.3, "non-prime fields"): an element is a polynomial
c_0 + c_1 x + ... + c_{n-1} x^{n-1} over F_p with code sum_j c_j p^j.  The
defining polynomial is f = x^n - (r_0 + r_1 x + ... + r_{n-1} x^{n-1}), stored
as r.  GF(4) uses the paper's x^2 + x + 1; the paper fixes no polynomial for
the other fields, and each one here is monic, irreducible and primitive (x
generates the multiplicative group), which the tests check.
"""
from __future__ import annotations

PRIMES = (2, 3, 5, 7)

# q: (p, n, r) with x^n = r_0 + r_1 x + ... (coefficients mod p)
EXTENSIONS = {
    4: (2, 2, (1, 1)),         # x^2 + x + 1
    8: (2, 3, (1, 1, 0)),      # x^3 + x + 1
    9: (3, 2, (1, 1)),         # x^2 + 2x + 2
    25: (5, 2, (3, 1)),        # x^2 + 4x + 2
    27: (3, 3, (2, 1, 0)),     # x^3 + 2x + 1
    49: (7, 2, (4, 1)),        # x^2 + 6x + 3
    125: (5, 3, (2, 2, 0)),    # x^3 + 3x + 3
}

FIELDS = PRIMES + tuple(sorted(EXTENSIONS))


def base(q: int) -> tuple[int, int]:
    """(p, n) with q = p^n."""
    if q in PRIMES:
        return q, 1
    if q in EXTENSIONS:
        p, n, _ = EXTENSIONS[q]
        return p, n
    raise ValueError("unsupported field size %r" % (q,))
