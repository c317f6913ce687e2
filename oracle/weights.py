"""RBF-FD Laplacian weights, one dense solve per stencil.  TEST INFRASTRUCTURE ONLY.

Sec. II, Eq. 1: (L u)(x_c) ~ sum_{p in N(x_c)} w_p u(p), with the weights of
the RBF-FD method; Sec. V fixes the basis: polyharmonic spline Phi(r) = r^3
augmented with all monomials of degree <= m (m in {2, 4, 6}), and L = lap (the
2D Laplacian, Sec. IV).

The weights solve the augmented (saddle-point) system of PHS+polynomial
RBF-FD, which the paper takes from its reference on RBF-FD and does not
print; the reading used here:

    [ Phi  P ] [ w      ]   [ L phi_j (x_c) ]
    [ P^T  0 ] [ lambda ] = [ L p_k   (x_c) ]

    Phi_jk = |x_j - x_k|^3                  (n x n)
    P_jk   = p_k(x_j), k over the monomials (n x s, s = (m+1)(m+2)/2)
    L phi_j (x_c) = lap |x - x_j|^3 at x = x_c = 9 |x_c - x_j|   (2D)
    L p_k (x_c)

The system is written in shifted and scaled coordinates xh = (x - x_c)/delta
with delta = the largest |x_j - x_c| in the stencil (for a nearest-neighbour
stencil, the distance to its n-th node).  r^3 is homogeneous of degree 3 and
the monomial space is closed under affine maps, so in exact arithmetic this
only rescales the unknowns: the Laplacian weights in the original coordinates
are w = wh / delta^2.  Monomials are in graded order
1, x, y, x^2, xy, y^2, x^3, x^2 y, ... (degree d lists x^(d-i) y^i, i = 0..d);
at xh = 0 only x^2 and y^2 have a nonzero Laplacian (2).

The solve is LAPACK's LU with partial pivoting (numpy.linalg.solve), applied
per stencil.  The system is singular when two stencil nodes coincide (two
identical rows and columns) or when P lacks full column rank (the nodes do
not determine the polynomials, e.g. all on one line); rank is read from the
singular values of P (smallest below 1e-12 of the largest: P's entries are
monomials of points in the unit disk).  Such stencils, and systems whose
solve fails or is not finite, get status 1.
"""

from __future__ import annotations

import numpy as np


def n_monomials(m: int) -> int:
    """s = (m+1)(m+2)/2 monomials of degree <= m in 2D."""
    return (m + 1) * (m + 2) // 2


def monomial_exponents(m: int) -> list:
    """(a, b) for the monomials x^a y^b in graded order."""
    return [(d - i, i) for d in range(m + 1) for i in range(d + 1)]


def _lap_monomial_at_origin(a: int, b: int) -> float:
    # lap x^a y^b = a(a-1) x^(a-2) y^b + b(b-1) x^a y^(b-2); at 0 only (2,0), (0,2) survive.
    return 2.0 if (a, b) in ((2, 0), (0, 2)) else 0.0


def local_system(xs: np.ndarray, m: int):
    """Augmented matrix and right-hand side for scaled stencil points.

    xs: (B, n, 2) stencil coordinates already shifted to the centre and scaled.
    Returns A (B, M, M) and rhs (B, M) with M = n + s.
    """
    B, n, _ = xs.shape
    ex = monomial_exponents(m)
    s = len(ex)
    M = n + s
    dx = xs[:, :, None, 0] - xs[:, None, :, 0]
    dy = xs[:, :, None, 1] - xs[:, None, :, 1]
    r = np.sqrt(dx * dx + dy * dy)
    A = np.zeros((B, M, M), dtype=np.float64)
    A[:, :n, :n] = r * r * r
    P = np.empty((B, n, s), dtype=np.float64)
    for k, (a, b) in enumerate(ex):
        P[:, :, k] = xs[:, :, 0] ** a * xs[:, :, 1] ** b
    A[:, :n, n:] = P
    A[:, n:, :n] = np.transpose(P, (0, 2, 1))
    rhs = np.empty((B, M), dtype=np.float64)
    rc = np.sqrt(xs[:, :, 0] * xs[:, :, 0] + xs[:, :, 1] * xs[:, :, 1])
    rhs[:, :n] = 9.0 * rc
    rhs[:, n:] = np.array([_lap_monomial_at_origin(a, b) for (a, b) in ex])[None, :]
    return A, rhs


def scaled_stencil(xy: np.ndarray, idx: np.ndarray, nodes: np.ndarray):
    """Shifted/scaled stencil coordinates (B, n, 2) and the scale delta (B,)."""
    return _scaled_rows(xy, idx[nodes], nodes)


def _scaled_rows(xy: np.ndarray, sten: np.ndarray, centres: np.ndarray):
    X = xy[sten.astype(np.int64)] - xy[centres][:, None, :]
    d2 = X[:, :, 0] * X[:, :, 0] + X[:, :, 1] * X[:, :, 1]
    delta = np.sqrt(d2.max(axis=1))
    return X / delta[:, None, None], delta


def weights(xy: np.ndarray, idx: np.ndarray, m: int, nodes=None, chunk: int = 2048):
    """Laplacian weights w (len(nodes), n) float64 and a per-node status (0 = ok).

    Row r holds the weights of stencil idx[nodes[r]] in the same order.
    Status 1 marks a stencil whose system is singular (e.g. coincident nodes).
    """
    idx = np.asarray(idx)
    if nodes is None:
        nodes = np.arange(idx.shape[0])
    nodes = np.asarray(nodes, dtype=np.int64)
    return weights_rows(xy, idx[nodes], nodes, m, chunk)


def weights_rows(xy: np.ndarray, sten: np.ndarray, centres: np.ndarray, m: int, chunk: int = 2048):
    """The same for explicit stencil rows: row r of `sten` is the stencil of
    node centres[r] (its weights approximate the Laplacian at that node)."""
    xy = np.asarray(xy, dtype=np.float64)
    sten = np.asarray(sten)
    centres = np.asarray(centres, dtype=np.int64)
    n = sten.shape[1]
    out = np.zeros((centres.size, n), dtype=np.float64)
    status = np.zeros(centres.size, dtype=np.int32)
    for s0 in range(0, centres.size, chunk):
        sel = slice(s0, s0 + chunk)
        xs, delta = _scaled_rows(xy, sten[sel], centres[sel])
        B = xs.shape[0]
        A, rhs = local_system(xs, m)
        # coincident nodes: an exactly zero distance off the diagonal
        dxx = xs[:, :, None, 0] - xs[:, None, :, 0]
        dyy = xs[:, :, None, 1] - xs[:, None, :, 1]
        off = ~np.eye(n, dtype=bool)[None]
        dup = ((dxx == 0.0) & (dyy == 0.0) & off).any(axis=(1, 2))
        sv = np.linalg.svd(A[:, :n, n:], compute_uv=False)
        dup |= ~(sv[:, -1] > 1e-12 * sv[:, 0])
        try:
            sol = np.linalg.solve(A, rhs[..., None])[..., 0]
            bad = ~np.isfinite(sol).all(axis=1)
        except np.linalg.LinAlgError:
            sol = np.zeros_like(rhs)
            bad = np.zeros(B, dtype=bool)
            for r in range(B):
                try:
                    sol[r] = np.linalg.solve(A[r], rhs[r])
                    bad[r] = not np.isfinite(sol[r]).all()
                except np.linalg.LinAlgError:
                    bad[r] = True
        bad = bad | dup
        out[sel] = sol[:, :n] / (delta * delta)[:, None]
        status[sel] = bad.astype(np.int32)
        out[sel][bad] = 0.0
    return out, status
