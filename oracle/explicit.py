"""The paper's explicit time loop and its data-size model.  TEST INFRASTRUCTURE ONLY.

Eq. 4 (Sec. IV): u_2 = u_1 + dt (f + lap u_1) on interior nodes, with lap
replaced by the RBF-FD weights; boundary nodes keep their Dirichlet values.

Sec. V, Table 1: the data copied to the GPU is N (4 + n) doubles and
N_i + N n 32-bit integers; setting N_i = N and equating the bytes to the L2
size gives the node count at which the working set fills L2.
"""

from __future__ import annotations

import numpy as np


def explicit_step(idx, w, is_dirichlet, f, u1, dt: float) -> np.ndarray:
    """One forward-Euler step of Eq. 4 (Dirichlet nodes unchanged)."""
    lap = np.einsum("ij,ij->i", w, u1[np.asarray(idx, dtype=np.int64)])
    dmask = np.asarray(is_dirichlet).astype(bool)
    return np.where(dmask, u1, u1 + dt * (f + lap))


def l2_estimate_nodes(cache_bytes: float, n: int) -> int:
    """N with 8 N (4 + n) + 4 (N + N n) = cache_bytes, rounded to the nearest node."""
    return int(round(cache_bytes / (8.0 * (4 + n) + 4.0 * (1 + n))))
