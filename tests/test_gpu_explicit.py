"""GPU tests of the explicit time loop (Sec. IV, Eq. 4) against the oracle's
forward-Euler step: several tiles of rows, the CUDA-graph replay path and
its remainder, the Dirichlet rows, the discrete steady state as a fixed
point, and sampled rows of a 1M-node step."""

import numpy as np
import pytest
import torch

import oracle
from fixtures import disk_nodes, manufactured

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _setup(h, m, n):
    d = disk_nodes(h)
    u, f, g = manufactured(d.xy)
    idx = oracle.knn(d.xy, n)
    w, _ = oracle.weights(d.xy, idx, m)
    return d, idx, w, f, g


@pytest.mark.parametrize("steps", [0, 1, 2, 63, 128, 129, 1000])
def test_explicit_steps_vs_oracle(lib, steps):
    from paper_2107_03632_gb300 import rbffd

    d, idx, w, f, g = _setup(0.04, 2, 12)
    rng = np.random.default_rng(7)
    u0 = rng.standard_normal(d.N)
    u0[d.is_dirichlet == 1] = g[d.is_dirichlet == 1]
    dt = 1e-5  # stable: dt |lap| well below 2 at h = 0.04
    ref = u0.copy()
    for _ in range(steps):
        ref = oracle.explicit_step(idx, w, d.is_dirichlet, f, ref, dt)
    loop = rbffd.ExplicitLoop(T(idx), T(w), T(d.is_dirichlet))
    assert loop.n_interior == int((d.is_dirichlet == 0).sum())
    u = T(u0)
    loop.run(T(f), u, dt, steps)
    got = u.cpu().numpy()
    assert np.array_equal(got[d.is_dirichlet == 1], u0[d.is_dirichlet == 1])
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= 1e-12, (steps, err)


def test_explicit_steady_state_is_a_fixed_point(lib):
    from paper_2107_03632_gb300 import rbffd

    d, idx, w, f, g = _setup(0.03, 4, 30)
    rp, col, val = oracle.assemble(idx, w, d.is_dirichlet)
    ust = oracle.solve_direct(rp, col, val, oracle.rhs(f, g, d.is_dirichlet))
    loop = rbffd.ExplicitLoop(T(idx), T(w), T(d.is_dirichlet))
    u = T(ust)
    loop.run(T(f), u, 1e-6, 200)
    assert np.abs(u.cpu().numpy() - ust).max() <= 1e-9 * np.abs(ust).max()


def test_explicit_rejects_out_of_range_index(lib):
    from paper_2107_03632_gb300 import rbffd

    d, idx, w, f, g = _setup(0.08, 2, 12)
    bad = idx.copy()
    bad[int(np.flatnonzero(d.is_dirichlet == 0)[3]), 5] = d.N + 7
    with pytest.raises(rbffd.RbffdError):
        rbffd.ExplicitLoop(T(bad), T(w), T(d.is_dirichlet))


def test_explicit_full_size_sampled_rows(lib):
    """1M nodes, m = 4, n = 30: one GPU step on the GPU's own stencils and
    weights; at sampled interior rows the oracle's stencil and weights
    (computed for those rows alone) give the same step."""
    from paper_2107_03632_gb300 import rbffd

    h, m, n = 1.7725e-3, 4, 30
    d = disk_nodes(h)
    u, f, g = manufactured(d.xy)
    xy = T(d.xy)
    idx = rbffd.rbffd_stencils(xy, n)
    w, st = rbffd.rbffd_weights(xy, idx, m)
    loop = rbffd.ExplicitLoop(idx, w, T(d.is_dirichlet))
    rng = np.random.default_rng(3)
    u0 = u + 1e-3 * rng.standard_normal(d.N)
    ug = T(u0)
    dt = 1e-7
    loop.run(T(f), ug, dt, 1)
    got = ug.cpu().numpy()
    rows = rng.choice(np.flatnonzero(d.is_dirichlet == 0), 200, replace=False)
    idx_o = oracle.knn_query(d.xy, n, rows)
    assert np.array_equal(idx.cpu().numpy()[rows], idx_o)
    w_o, _ = oracle.weights(d.xy, _scatter(idx_o, rows, d.N, n), m, nodes=rows)
    terms = w_o * u0[idx_o.astype(np.int64)]
    ref = u0[rows] + dt * (f[rows] + terms.sum(axis=1))
    # weights agree to 1e-9 of the stencil's largest weight (the weights'
    # parity bar): the step may differ by dt * 1e-9 * max|w| * sum |u|, plus
    # rounding
    uu = np.abs(u0[idx_o.astype(np.int64)]).sum(axis=1)
    bound = dt * 1e-9 * np.abs(w_o).max(axis=1) * uu + 4e-16 * np.abs(ref)
    assert (np.abs(got[rows] - ref) <= bound).all()


def _scatter(idx_rows, rows, N, n):
    full = np.zeros((N, n), dtype=np.int32)
    full[rows] = idx_rows
    return full
