"""Direct solve of the assembled system and its adjoint.  TEST INFRASTRUCTURE ONLY.

Sec. VI names the implicit solution of the Poisson problem as the next step
after the paper's explicit loop; its plain definition is u = A^{-1} b with A
and b from `oracle.assemble`.  The oracle computes it with a direct solver:
dense LU with partial pivoting (LAPACK via numpy) for small systems, SuperLU
(scipy.sparse.linalg.splu) otherwise.

Adjoint gradient of a loss L(u) with u = A^{-1} b(f, g):
    A^T lambda = dL/du,   dL/df_i = -lambda_i (interior rows, since b_i = -f_i),
                          dL/dg_i = +lambda_i (Dirichlet rows, since b_i = g_i),
and zero elsewhere.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .assemble import assemble, rhs, to_scipy
from .knn import knn
from .weights import weights

DENSE_LIMIT = 3000


def solve_direct(row_ptr, col, val, b, transpose: bool = False) -> np.ndarray:
    """x with A x = b (or A^T x = b)."""
    N = row_ptr.size - 1
    A = to_scipy(row_ptr, col, val, N)
    if transpose:
        A = A.T
    if N <= DENSE_LIMIT:
        return np.linalg.solve(A.toarray(), b)
    lu = spla.splu(A.tocsc(), permc_spec="COLAMD")
    return lu.solve(np.asarray(b, dtype=np.float64))


def adjoint_gradient(row_ptr, col, val, is_dirichlet, dLdu):
    """(dL/df, dL/dg) for L(u), u = A^{-1} b, from the adjoint solve A^T lambda = dL/du."""
    lam = solve_direct(row_ptr, col, val, dLdu, transpose=True)
    dmask = np.asarray(is_dirichlet).astype(bool)
    return np.where(dmask, 0.0, -lam), np.where(dmask, lam, 0.0), lam


def poisson_solve(xy, is_dirichlet, f, g, m: int, n: int):
    """Full pipeline on the CPU: stencils, weights, assembly, direct solve."""
    idx = knn(xy, n)
    w, status = weights(xy, idx, m)
    if status.any():
        raise np.linalg.LinAlgError("singular stencil system")
    row_ptr, col, val = assemble(idx, w, is_dirichlet)
    b = rhs(f, g, is_dirichlet)
    return solve_direct(row_ptr, col, val, b), (idx, w, row_ptr, col, val, b)
