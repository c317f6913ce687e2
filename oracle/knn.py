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


def knn_grid(xy: np.ndarray, n: int, queries=None, chunk: int = 16384) -> np.ndarray:
    """The same stencils as `knn_query` (identical rows, the same (d^2, j)
    order and keys), found among the nodes of a block of grid cells around each
    query instead of all N nodes: for large node sets, where the brute force
    costs O(N) per query.

    Nodes are binned into square cells of side c.  A query in cell (cx, cy)
    first takes every node of the (2R+1) x (2R+1) block of cells around it.
    Any node outside that block lies farther than R c from the query, so when
    the n-th smallest distance among the block's nodes is below R c, every
    node at that distance or closer is in the block and the block's first n
    keys are the brute force's first n.  Queries that miss this bound are
    redone with R + 1 (and, past a few rings, by brute force)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    N = xy.shape[0]
    if n > N:
        raise ValueError("stencil size n exceeds the number of nodes")
    if queries is None:
        queries = np.arange(N)
    queries = np.asarray(queries, dtype=np.int64)
    lo = xy.min(axis=0)
    span = float(max((xy.max(axis=0) - lo).max(), 1e-300))
    # cells of about one node each (bounding-box density)
    c = span / max(1.0, np.floor(np.sqrt(N)))
    nc = int(np.floor(span / c)) + 1
    cxy = np.minimum(np.floor((xy - lo) / c).astype(np.int64), nc - 1)
    key = cxy[:, 1] * nc + cxy[:, 0]
    order = np.argsort(key, kind="stable")
    start = np.searchsorted(key[order], np.arange(nc * nc + 1))
    # first ring whose disc of radius R c holds about 2n nodes at that density
    R0 = max(1, int(np.ceil(np.sqrt(2.0 * n / np.pi))))
    out = np.empty((queries.size, n), dtype=np.int32)
    todo = np.arange(queries.size)
    R = R0
    while todo.size:
        if R > R0 + 3:  # unusual clustering: the definition itself
            out[todo] = knn_query(xy, n, queries[todo])
            break
        retry = []
        for s0 in range(0, todo.size, chunk):
            sel = todo[s0 : s0 + chunk]
            q = queries[sel]
            qc = cxy[q]
            # (2R+1) row segments per query: cells (cx-R .. cx+R, cy + dy),
            # contiguous in the cell-sorted order
            dys = np.arange(-R, R + 1)
            cy = qc[:, 1:2] + dys[None, :]
            x0 = np.clip(qc[:, 0:1] - R, 0, nc - 1)
            x1 = np.clip(qc[:, 0:1] + R, 0, nc - 1)
            valid = (cy >= 0) & (cy < nc)
            cyc = np.clip(cy, 0, nc - 1)
            a = start[cyc * nc + x0]
            b = start[cyc * nc + x1 + 1]
            ln = np.where(valid, b - a, 0)
            cum = np.cumsum(ln, axis=1)
            L = max(int(cum[:, -1].max()), n)  # at least n slots (missing ones: infinite keys)
            pos = np.arange(L)
            seg = (pos[None, :, None] >= cum[:, None, :]).sum(axis=2)  # segment of each slot
            inside = pos[None, :] < cum[:, -1:]
            segc = np.minimum(seg, 2 * R)
            off = pos[None, :] - (np.take_along_axis(cum, segc, axis=1) - np.take_along_axis(ln, segc, axis=1))
            cand = order[np.where(inside, np.take_along_axis(a, segc, axis=1) + off, 0)]
            dx = xy[cand, 0] - xy[q, 0][:, None]
            dy = xy[cand, 1] - xy[q, 1][:, None]
            d2 = dx * dx + dy * dy
            d2 = np.where(inside, d2, np.inf)
            cj = np.where(inside, cand, np.iinfo(np.int64).max)
            srt = np.lexsort((cj, d2), axis=1)[:, :n]
            dn2 = np.take_along_axis(d2, srt[:, n - 1 : n], axis=1)[:, 0]
            ok = dn2 < (R * c * (1.0 - 1e-9)) ** 2
            out[sel[ok]] = np.take_along_axis(cand, srt, axis=1)[ok]
            retry.append(sel[~ok])
        todo = np.concatenate(retry) if retry else np.zeros(0, dtype=np.int64)
        R += 1
    return out
