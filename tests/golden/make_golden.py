"""Writes the closed-form golden fixtures in this folder (uses sympy only, never the
oracle or the GPU library).

* toeplitz121_n8.txt: eigenvalues 2 - 2 cos(k pi / 9), k = 1..8, of tridiag(1, 2, 1)
  of order 8 (the matrix of Example 2 and the Toeplitz-type matrix of Example 3),
  to 30 significant digits.
* clement_n7.txt: eigenvalues of the Clement-type matrix of Example 3 (zero diagonal,
  off-diagonal sqrt(i (7 - i)), i = 1..6): the integers -6, -4, ..., 6.
"""
import os

import sympy as sp

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    n = 8
    with open(os.path.join(HERE, "toeplitz121_n8.txt"), "w") as f:
        f.write("# tridiag(1,2,1), n=8: lambda_k = 2 - 2 cos(k pi/(n+1)) (Example 2 / Example 3 matrix)\n")
        for k in range(1, n + 1):
            f.write(sp.N(2 - 2 * sp.cos(k * sp.pi / (n + 1)), 30).__str__() + "\n")
    m = 7
    t = sp.zeros(m, m)
    for i in range(1, m):
        t[i - 1, i] = t[i, i - 1] = sp.sqrt(i * (m - i))
    ev = sorted(sp.Matrix(t).eigenvals().keys(), key=lambda x: float(x))
    with open(os.path.join(HERE, "clement_n7.txt"), "w") as f:
        f.write("# Clement-type matrix of Example 3, order 7 (off-diagonal sqrt(i(7-i))), exact eigenvalues\n")
        for v in ev:
            f.write(str(sp.nsimplify(v)) + "\n")


if __name__ == "__main__":
    main()
