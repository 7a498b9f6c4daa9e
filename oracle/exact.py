"""Exact rational solution of Eq. 1 by Gauss-Jordan elimination (brute force).

TEST INFRASTRUCTURE ONLY: used by the tests and by the script that writes the
golden fixtures under tests/golden/.  Not part of the product path.

This is the plain definition of the result (Eq. 1 of arXiv 2310.17556):
form the dense m x m matrix A = S^T S + lambda I in exact rational arithmetic
and solve A x = v by Gauss-Jordan elimination with ``fractions.Fraction``.
It does not follow Algorithm 1 at all, which is what makes it a pin for the
FP64 oracle (``oracle.alg1``) and, through the fixtures, for the GPU path.
Only meant for tiny m (m <= 8): the cost is O(m^3) Fraction operations.
"""

from __future__ import annotations

from fractions import Fraction

__all__ = ["solve_dense_exact"]


def solve_dense_exact(S, v, lam):
    """Return x (list of Fractions) with (S^T S + lam I) x = v, exactly.

    S: list of n rows, each a list of m rationals (ints/Fractions/str).
    v: list of m rationals.  lam: a positive rational.
    """
    S = [[Fraction(e) for e in row] for row in S]
    v = [Fraction(e) for e in v]
    lam = Fraction(lam)
    if lam <= 0:
        raise ValueError("lambda must be positive")
    n = len(S)
    m = len(v)
    if any(len(row) != m for row in S):
        raise ValueError("S rows must have length m")
    # A = S^T S + lam I, entry (p, q) = sum_i S[i][p] S[i][q] + lam [p == q]
    A = [[sum((S[i][p] * S[i][q] for i in range(n)), Fraction(0)) + (lam if p == q else 0)
          for q in range(m)] for p in range(m)]
    aug = [A[p] + [v[p]] for p in range(m)]
    for col in range(m):
        piv = next((r for r in range(col, m) if aug[r][col] != 0), None)
        if piv is None:
            raise ZeroDivisionError("singular system")
        aug[col], aug[piv] = aug[piv], aug[col]
        p = aug[col][col]
        aug[col] = [e / p for e in aug[col]]
        for r in range(m):
            if r != col and aug[r][col] != 0:
                f = aug[r][col]
                aug[r] = [a - f * b for a, b in zip(aug[r], aug[col])]
    return [aug[p][m] for p in range(m)]
