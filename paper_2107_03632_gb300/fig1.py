"""The paper's Fig. 1 case, headless: Poisson on the unit disk with
u = sin(pi x) sin(pi y), m = 2, n = 15 and N = 1027 nodes (Sec. III), solved
on the GPU; writes "x y u" per node to a text file (no plotting).

    python -m paper_2107_03632_gb300.fig1 out.txt [fp64|mixed] [mg|none]

The node set is the seeded jittered disk of the repository's fixtures at
h = 0.05692 (N = 1027).
"""

from __future__ import annotations

import os
import sys

import numpy as np
import torch

from .pipeline import poisson_solve

H_FIG1 = 0.05692
M_FIG1, N_FIG1 = 2, 15


def fig1(path: str, precision: str = "fp64", precond: str | None = None, device: str = "cuda:0"):
    """Solves the Fig. 1 case and writes x, y, u; returns (xy, u, info)."""
    try:
        from fixtures import disk_nodes, manufactured
    except ImportError:  # run from elsewhere: the fixtures sit at the repository root
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        from fixtures import disk_nodes, manufactured
    d = disk_nodes(H_FIG1)
    _, f, g = manufactured(d.xy)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
    u, info, _ = poisson_solve(T(d.xy), T(d.is_dirichlet), T(f), T(g), M_FIG1, N_FIG1, precision=precision,
                               precond=precond)
    uh = u.cpu().numpy()
    np.savetxt(path, np.column_stack([d.xy, uh]), fmt="%.17g", header=f"x y u  (N={d.N}, m={M_FIG1}, n={N_FIG1})")
    return d.xy, uh, info


def main(argv=None) -> int:
    argv = sys.argv[1:] if argv is None else argv
    if not argv:
        print(__doc__)
        return 2
    precision = argv[1] if len(argv) > 1 else "fp64"
    precond = (argv[2] if len(argv) > 2 else "none")
    _, _, info = fig1(argv[0], precision, None if precond == "none" else precond)
    print(info)
    return 0 if info["status"] == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
