"""Exact Laplacian weights of unisolvent stencils (n = s), for the tests.

When a stencil has exactly s = (m+1)(m+2)/2 nodes and P is invertible, the
polynomial block of the augmented system, sum_j w_j p_k(x_j - x_c) =
lap p_k(0) for every monomial of degree <= m, fixes the weights on its own
(Sec. II Eq. 1 with the basis of Sec. V; the r^3 part drops out).  Shifted
coordinates X = x_j - x_c are taken as the doubles that both the oracle and
the GPU form; as rationals they define the system exactly, which is solved
here in exact rational arithmetic (fractions) by Gaussian elimination.  The
shift is kept and the scaling left out: the weights of the Laplacian are
invariant under it in exact arithmetic.
"""

from fractions import Fraction

import numpy as np


def exact_weights(xy: np.ndarray, sten: np.ndarray, centre: int, m: int) -> np.ndarray:
    ex = [(d - i, i) for d in range(m + 1) for i in range(d + 1)]
    s = len(ex)
    assert sten.size == s
    X = [(Fraction(float(xy[j, 0] - xy[centre, 0])), Fraction(float(xy[j, 1] - xy[centre, 1]))) for j in sten]
    # rows k: sum_j p_k(X_j) w_j = lap p_k(0)
    M = [[X[j][0] ** a * X[j][1] ** b for j in range(s)] + [Fraction(2 if (a, b) in ((2, 0), (0, 2)) else 0)]
         for (a, b) in ex]
    for c in range(s):
        piv = next(r for r in range(c, s) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(s):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return np.array([float(M[j][s]) for j in range(s)])
