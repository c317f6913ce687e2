"""The paper's Fig. 1 case (Sec. III: unit disk, u = sin(pi x) sin(pi y),
m = 2, n = 15, N = 1027) as a headless regression: the GPU solution written
to a file matches the oracle's direct solve to the solution bar, and the
manufactured solution to the discretisation error."""

import numpy as np
import pytest

import oracle
from fixtures import disk_nodes, manufactured

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,precond", [("fp64", None), ("mixed", None), ("fp64", "mg"), ("mixed", "mg")])
def test_fig1_case(lib, tmp_path, precision, precond):
    from paper_2107_03632_gb300 import fig1

    path = tmp_path / "fig1_u.txt"
    xy, u, info = fig1.fig1(str(path), precision, precond)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    d = disk_nodes(fig1.H_FIG1)
    assert d.N == 1027 and np.array_equal(xy, d.xy)
    back = np.loadtxt(path)
    assert back.shape == (1027, 3) and np.array_equal(back[:, 2], u) and np.array_equal(back[:, :2], d.xy)
    u_ex, f, g = manufactured(d.xy)
    ref, _ = oracle.poisson_solve(d.xy, d.is_dirichlet, f, g, fig1.M_FIG1, fig1.N_FIG1)
    assert np.abs(u - ref).max() / np.abs(ref).max() <= 1e-8
    # second-order stencils on ~0.06 spacing: the error against sin(pi x) sin(pi y)
    # is that of the discretisation, the same on both sides
    err = np.abs(u - u_ex).max()
    assert err <= 2e-2 and abs(err - np.abs(ref - u_ex).max()) <= 1e-8
