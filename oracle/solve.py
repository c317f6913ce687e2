"""Solves of the assembled system and its adjoint.  TEST INFRASTRUCTURE ONLY.

Sec. VI names the implicit solution of the Poisson problem as the next step
after the paper's explicit loop; its plain definition is u = A^{-1} b with A
and b from `oracle.assemble`.  The oracle computes it with a direct solver:
dense LU with partial pivoting (LAPACK via numpy) for small systems, SuperLU
(scipy.sparse.linalg.splu) otherwise.

For node sets where a direct factorisation of A does not fit (millions of
nodes at m = 6), `solve_refined` reaches the same u by iterative refinement:
the residual b - A x is formed with every product and sum in extended
precision (numpy.longdouble), and each correction A d = r is solved by
restarted GMRES right-preconditioned with a SuperLU factorisation of a
cheaper operator M (the caller's choice; in the tests, the degree-2,
12-node RBF-FD Laplacian of the same nodes).  M only changes how fast the
corrections converge; the fixed point is A^{-1} b.

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


def residual_extended(row_ptr, col, val, x, b, transpose: bool = False, chunk_nnz: int = 1 << 23) -> np.ndarray:
    """b - A x (or b - A^T x) with the products a_ij x_j and their sums in
    numpy.longdouble (a 64-bit significand on x86, 113 on aarch64), rounded to
    float64 at the end.  Every row of A has at least one entry."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    N = row_ptr.size - 1
    if transpose:
        A = to_scipy(row_ptr, col, val, N).T.tocsr()
        row_ptr, col, val = A.indptr.astype(np.int64), A.indices, A.data
    xl = np.asarray(x, dtype=np.float64).astype(np.longdouble)
    r = np.empty(N, dtype=np.float64)
    row = 0
    while row < N:
        end = int(np.searchsorted(row_ptr, row_ptr[row] + chunk_nnz, side="right")) - 1
        end = min(max(end, row + 1), N)
        a, e = int(row_ptr[row]), int(row_ptr[end])
        prod = np.asarray(val[a:e], dtype=np.float64).astype(np.longdouble) * xl[col[a:e]]
        acc = np.add.reduceat(prod, row_ptr[row:end] - a)
        r[row:end] = (np.asarray(b[row:end], dtype=np.float64).astype(np.longdouble) - acc).astype(np.float64)
        row = end
    return r


def gmres_right(matvec, psolve, b, tol: float, restart: int = 60, max_cycles: int = 200):
    """Restarted GMRES for A d = b, right-preconditioned: d = M^{-1} z with z
    from the Krylov space of A M^{-1}, minimising |b - A d|_2 (Saad and Schultz
    1986; Givens rotations on the Hessenberg matrix, Gram-Schmidt applied twice).
    Stops when |b - A d|_2 <= tol |b|_2.  Returns (d, iterations)."""
    N = b.size
    d = np.zeros(N)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return d, 0
    its = 0
    for _ in range(max_cycles):
        r = b - matvec(d)
        beta = float(np.linalg.norm(r))
        if beta <= tol * bnorm:
            break
        V = np.empty((restart + 1, N))
        V[0] = r / beta
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        gvec = np.zeros(restart + 1)
        gvec[0] = beta
        k = 0
        for j in range(restart):
            wv = matvec(psolve(V[j]))
            for _pass in range(2):
                hcol = V[: j + 1] @ wv
                wv -= hcol @ V[: j + 1]
                H[: j + 1, j] += hcol
            H[j + 1, j] = float(np.linalg.norm(wv))
            V[j + 1] = wv / H[j + 1, j] if H[j + 1, j] > 0 else 0.0
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = float(np.hypot(H[j, j], H[j + 1, j]))
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            k = j + 1
            its += 1
            if abs(gvec[j + 1]) <= tol * bnorm:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (gvec[i] - H[i, i + 1 : k] @ y[i + 1 :]) / H[i, i]
        d = d + psolve(y @ V[:k])
    return d, its


def solve_refined(row_ptr, col, val, b, precond=None, transpose: bool = False, inner_tol: float = 1e-6,
                  max_refine: int = 8, restart: int = 60):
    """x with A x = b (A^T x = b) by iterative refinement in extended
    precision: r = b - A x (residual_extended), A d = r by gmres_right with
    M^{-1} from SuperLU, x += d, until the correction is below four units in
    the last place of x.  precond: CSR arrays (row_ptr, col, val) of M (M^T
    is used for the transpose); None: M = A (SuperLU of A itself, i.e.
    classical iterative refinement of the direct solve).  Returns (x, info)."""
    N = np.asarray(row_ptr).size - 1
    A = to_scipy(row_ptr, col, val, N)
    Mm = to_scipy(*precond, N) if precond is not None else A
    if transpose:
        A, Mm = A.T.tocsr(), Mm.T
    # diagonal pivots keep the fill-reducing order of the symmetrised pattern:
    # interior rows are diagonally dominant, and a Dirichlet row is a unit
    # row (its column's other entries are eliminated without fill or growth),
    # whereas row exchanges toward those columns' large interior entries
    # multiplied the fill and the factorisation time tenfold here
    lu = spla.splu(Mm.tocsc(), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0)
    x = np.zeros(N)
    b = np.asarray(b, dtype=np.float64)
    hist = []
    for _ in range(max_refine):
        r = residual_extended(row_ptr, col, val, x, b, transpose=transpose)
        d, its = gmres_right(A.dot, lu.solve, r, inner_tol, restart=restart)
        x = x + d
        hist.append({"res": float(np.linalg.norm(r) / np.linalg.norm(b)), "gmres_its": its,
                     "corr": float(np.abs(d).max() / max(np.abs(x).max(), 1e-300))})
        if hist[-1]["corr"] <= 4 * np.finfo(np.float64).eps:
            break
    r = residual_extended(row_ptr, col, val, x, b, transpose=transpose)
    return x, {"refinements": hist, "rel_residual": float(np.linalg.norm(r) / np.linalg.norm(b))}


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
