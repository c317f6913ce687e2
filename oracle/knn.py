"""Brute-force stencil (support) selection.  TEST INFRASTRUCTURE ONLY.

Sec. II (Eq. 1) approximates an operator at x from the values at N(x), the
set of neighbouring nodes; Sec. V takes N(x) to be the n nodes nearest to x.
Reading used here (the paper leaves both points open):

* the node x itself belongs to its own support (distance 0, listed first);
* candidates are ordered by the key (d^2, j), where d^2 is
  (x_j - x)*(x_j - x) + (y_j - y)*(y_j - y) with each product rounded to
  double and then added (no fused multiply-add), and j is the caller's node
  index, so equal distances are broken by the smaller index.

The stencil of node i is the first n entries of that order.
"""

from __future__ import annotations

import numpy as np


def _sqdist(xy: np.ndarray, q: np.ndarray) -> np.ndarray:
    # (B, N) squared distances; numpy rounds every product and sum separately.
    dx = xy[None, :, 0] - q[:, None, 0]
    dy = xy[None, :, 1] - q[:, None, 1]
    return dx * dx + dy * dy


def knn_query(xy: np.ndarray, n: int, queries: np.ndarray, chunk: int = 0) -> np.ndarray:
    """Stencils of the nodes listed in `queries` (indices into xy): (len(queries), n) int32."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    N = xy.shape[0]
    if n > N:
        raise ValueError("stencil size n exceeds the number of nodes")
    queries = np.asarray(queries, dtype=np.int64)
    out = np.empty((queries.size, n), dtype=np.int32)
    if chunk <= 0:
        chunk = max(1, min(queries.size, (1 << 21) // max(N, 1)))
    jidx = np.arange(N, dtype=np.int64)
    for s in range(0, queries.size, chunk):
        q = queries[s : s + chunk]
        d2 = _sqdist(xy, xy[q])
        for r in range(q.size):
            row = d2[r]
            # every index whose distance is <= the n-th smallest distance
            kth = np.partition(row, n - 1)[n - 1]
            cand = np.nonzero(row <= kth)[0]
            order = np.lexsort((jidx[cand], row[cand]))  # by d^2, then by index
            out[s + r] = cand[order[:n]]
    return out


def knn(xy: np.ndarray, n: int) -> np.ndarray:
    """Stencils of every node: (N, n) int32, row i lists node i's n nearest nodes."""
    return knn_query(xy, n, np.arange(xy.shape[0]))
