"""Writes lambda_grid.txt: points of the SURE threshold grid
lambda_k = k sqrt(2 ln N) / (K - 1) (the universal threshold of Donoho and
Johnstone, 1994, as the top of a uniform K-point grid), evaluated with
Python's decimal module at 40 significant digits, independently of numpy
and of the oracle.

Run from the repository root: python tests/golden/make_lambda_grid.py
"""

import os
from decimal import Decimal, getcontext

ROWS = [(675840, 64, 63), (675840, 64, 1), (675840, 64, 23), (4096, 64, 63), (4096, 64, 1)]


def grid_point(N: int, K: int, k: int) -> Decimal:
    getcontext().prec = 60
    top = (Decimal(2) * Decimal(N).ln()).sqrt()
    v = Decimal(k) * top / Decimal(K - 1)
    getcontext().prec = 40
    return +v


def main() -> None:
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lambda_grid.txt")
    with open(path, "w") as f:
        f.write("# Threshold grid lambda_k = k * sqrt(2 ln N) / (K - 1) (the universal\n"
                "# threshold of Donoho and Johnstone, 1994, as the top of a uniform K-point\n"
                "# grid), evaluated by tests/golden/make_lambda_grid.py with Python's decimal\n"
                "# module at 40 significant digits (Decimal(N).ln(), then .sqrt()),\n"
                "# independently of numpy.\n"
                "# columns: N K k lambda_k\n")
        for N, K, k in ROWS:
            f.write(f"{N} {K} {k} {grid_point(N, K, k)}\n")


if __name__ == "__main__":
    main()
