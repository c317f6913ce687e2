"""Discrete Poisson operator with Dirichlet rows.  TEST INFRASTRUCTURE ONLY.

Sec. IV, Eqs. 2-3: du/dt - lap u = f in the disk, u = g on its boundary.  At
steady state (the implicit solve named in Sec. VI) the interior equations are
-lap u = f, i.e. sum_j w_ij u_j = -f_i with the RBF-FD Laplacian weights of
node i, and each boundary node carries the Dirichlet equation u_i = g_i.

Reading: the matrix rows keep the sign of the Laplacian (+w) and the
right-hand side carries -f, so A is the discrete Laplacian on interior rows
and the identity on Dirichlet rows.  Columns of a row are in stencil order.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def assemble(idx: np.ndarray, w: np.ndarray, is_dirichlet: np.ndarray):
    """CSR arrays (row_ptr int64 (N+1,), col int32 (nnz,), val float64 (nnz,))."""
    idx = np.asarray(idx)
    N, n = idx.shape
    dir_mask = np.asarray(is_dirichlet).astype(bool)
    row_len = np.where(dir_mask, 1, n).astype(np.int64)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(row_len)
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    for i in range(N):
        a = row_ptr[i]
        if dir_mask[i]:
            col[a] = i
            val[a] = 1.0
        else:
            col[a : a + n] = idx[i]
            val[a : a + n] = w[i]
    return row_ptr, col, val


def to_scipy(row_ptr, col, val, N: int):
    """scipy.sparse CSR view of the arrays (no duplicate summation needed:
    the columns of one stencil are distinct nodes)."""
    return sp.csr_matrix((val, col, row_ptr), shape=(N, N))


def rhs(f: np.ndarray, g: np.ndarray, is_dirichlet: np.ndarray) -> np.ndarray:
    """b_i = -f_i on interior rows, g_i on Dirichlet rows."""
    dir_mask = np.asarray(is_dirichlet).astype(bool)
    return np.where(dir_mask, g, -f).astype(np.float64)
