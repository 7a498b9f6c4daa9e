"""Write the exact-rational fixtures in this folder (calls only ``oracle.exact``).

Each fixture is a tiny instance of Eq. 1 of arXiv 2310.17556,
(S^T S + lambda I) x = v, with small-integer S and v and a rational lambda,
solved exactly by Gauss-Jordan elimination over the rationals
(``oracle.exact.solve_dense_exact``, the plain definition of the result).

Run from the repository root:  python tests/golden/make_golden.py
"""

import json
import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.exact import solve_dense_exact  # noqa: E402

CASES = [
    # name, S (n rows of m), v (m), lambda
    ("n1_m3", [[1, -2, 2]], [3, 0, -1], "1/2"),
    ("n2_m4", [[1, 0, 2, -1], [0, 3, -1, 1]], [1, 2, 3, 4], "1/10"),
    ("n3_m5", [[2, -1, 0, 1, 3], [1, 1, -2, 0, 1], [0, 2, 1, -1, -2]], [5, -3, 2, 0, 1], "3/1000"),
    ("n3_m3_square", [[4, 1, -1], [2, -3, 1], [1, 0, 5]], [1, -1, 2], "1/4"),
    ("n4_m2_tall", [[1, 2], [-1, 1], [3, 0], [2, -2]], [7, -5], "2"),
]


def main():
    for name, S, v, lam in CASES:
        x = solve_dense_exact(S, v, Fraction(lam))
        doc = {
            "cite": "arXiv 2310.17556 Eq. 1: (S^T S + lambda I) x = v; exact rational solution by Gauss-Jordan",
            "n": len(S),
            "m": len(v),
            "S": S,
            "v": v,
            "lambda": lam,
            "x": [str(e) for e in x],
        }
        with open(os.path.join(HERE, f"eq1_exact_{name}.json"), "w") as f:
            json.dump(doc, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main()
