"""GPU tests of the multigrid-preconditioned solve.

The preconditioner changes how the solution is reached, not what it is: the
solution must match the oracle's direct solve to 1e-8 (relative max-norm) at
relative residual 1e-10, in FP64 and with the float32 V-cycle, and the
iteration count must stay small and flat as the node set is refined.
"""

import numpy as np
import pytest
import torch

import oracle
from fixtures import disk_nodes, manufactured
from oracle.assemble import to_scipy

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _system(h, m, n):
    d = disk_nodes(h)
    u, f, g = manufactured(d.xy)
    idx = oracle.knn(d.xy, n)
    w, _ = oracle.weights(d.xy, idx, m)
    rp, col, val = oracle.assemble(idx, w, d.is_dirichlet)
    b = oracle.rhs(f, g, d.is_dirichlet)
    return d, idx, w, rp, col, val, b


@pytest.mark.parametrize("h,m,n", [(0.04, 2, 12), (0.03, 4, 30), (0.05, 6, 56), (0.015, 2, 12)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mg_solve_vs_oracle(lib, h, m, n, precision):
    from paper_2107_03632_gb300 import rbffd

    d, idx, w, rp, col, val, b = _system(h, m, n)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    A = rbffd.rbffd_assemble(T(idx), T(w), mask, want_f32=True)
    mg = rbffd.Multigrid(xy, mask, A)
    lv = mg.levels()
    assert lv[0] == d.N and len(lv) >= 1
    assert all(lv[k + 1] <= lv[k] // 2 for k in range(len(lv) - 1))
    assert lv[-1] <= 128
    x, info = rbffd.rbffd_solve(A, T(b), opts=rbffd.make_opts(tol=1e-10, precision=precision, mg=mg))
    x = x.cpu().numpy()
    ref = oracle.solve_direct(rp, col, val, b)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    As = to_scipy(rp, col, val, d.N)
    assert np.linalg.norm(b - As @ x) / np.linalg.norm(b) <= 1e-10
    assert np.abs(x - ref).max() / np.abs(ref).max() <= 1e-8
    assert info["iters"] <= 60, info


def test_mg_single_level_is_exact_inverse(lib):
    """N <= 128: the hierarchy is the dense inverse alone; BiCGSTAB then needs
    one or two iterations."""
    from paper_2107_03632_gb300 import rbffd

    d, idx, w, rp, col, val, b = _system(0.18, 2, 12)
    assert d.N <= 128
    xy, mask = T(d.xy), T(d.is_dirichlet)
    A = rbffd.rbffd_assemble(T(idx), T(w), mask, want_f32=True)
    mg = rbffd.Multigrid(xy, mask, A)
    assert mg.levels() == [d.N]
    x, info = rbffd.rbffd_solve(A, T(b), opts=rbffd.make_opts(tol=1e-10, mg=mg))
    ref = oracle.solve_direct(rp, col, val, b)
    assert info["status"] == 0 and info["iters"] <= 3
    assert np.abs(x.cpu().numpy() - ref).max() / np.abs(ref).max() <= 1e-8


def test_mg_iterations_flat_under_refinement(lib):
    """Jacobi-BiCGSTAB iterations grow like 1/h; with the V-cycle they stay flat."""
    from paper_2107_03632_gb300 import rbffd

    its = []
    for h in (0.02, 0.01, 0.005):
        d = disk_nodes(h)
        u, f, g = manufactured(d.xy)
        xy, mask = T(d.xy), T(d.is_dirichlet)
        op_idx = rbffd.rbffd_stencils(xy, 30)
        wgt, st = rbffd.rbffd_weights(xy, op_idx, 4)
        A = rbffd.rbffd_assemble(op_idx, wgt, mask, want_f32=True)
        b = rbffd.rbffd_rhs(T(f), T(g), mask)
        mg = rbffd.Multigrid(xy, mask, A)
        x, info = rbffd.rbffd_solve(A, b, opts=rbffd.make_opts(tol=1e-10, precision="mixed", mg=mg))
        assert info["status"] == 0
        its.append(info["iters"])
    assert max(its) <= 40 and its[-1] <= 2 * its[0] + 5, its


def test_mg_deterministic(lib):
    from paper_2107_03632_gb300 import rbffd

    d, idx, w, rp, col, val, b = _system(0.02, 4, 30)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    A = rbffd.rbffd_assemble(T(idx), T(w), mask, want_f32=True)
    res = []
    for _ in range(2):
        mg = rbffd.Multigrid(xy, mask, A)
        for prec in ("fp64", "mixed"):
            x, info = rbffd.rbffd_solve(A, T(b), opts=rbffd.make_opts(precision=prec, mg=mg))
            res.append((x.clone(), info["iters"], mg.levels()))
    assert torch.equal(res[0][0], res[2][0]) and res[0][1] == res[2][1] and res[0][2] == res[2][2]
    assert torch.equal(res[1][0], res[3][0]) and res[1][1] == res[3][1]


def test_mg_rejects_mismatched_hierarchy(lib):
    from paper_2107_03632_gb300 import rbffd

    d1, idx1, w1, *_ = _system(0.04, 2, 12)
    d2, idx2, w2, rp, col, val, b = _system(0.05, 2, 12)
    A1 = rbffd.rbffd_assemble(T(idx1), T(w1), T(d1.is_dirichlet))
    A2 = rbffd.rbffd_assemble(T(idx2), T(w2), T(d2.is_dirichlet))
    mg = rbffd.Multigrid(T(d1.xy), T(d1.is_dirichlet), A1)  # built without A32: FP64 V-cycle only
    _, info = rbffd.rbffd_solve(A2, T(b), opts=rbffd.make_opts(mg=mg), raise_on_error=False)
    assert info["status_code"] == 1
    _, info = rbffd.rbffd_solve(A1, torch.ones(d1.N, dtype=torch.float64, device=DEV),
                                opts=rbffd.make_opts(precision="mixed", mg=mg), raise_on_error=False)
    assert info["status_code"] == 1


def test_mg_full_size_sampled_residual(lib):
    """1M nodes, m = 4, n = 30, the bench's launch configuration (multigrid,
    float32 V-cycle): the oracle cannot solve the system at this size, but it
    can recompute sampled rows of A from their own stencils and weights; on
    those rows |b_i - (A u)_i| must stay within the solve's bound
    1e-10 |b|_2 plus what the weights' parity bar (1e-9 of a stencil's
    largest weight) allows."""
    from paper_2107_03632_gb300 import rbffd

    h, m, n = 1.7725e-3, 4, 30
    d = disk_nodes(h)
    u_ex, f, g = manufactured(d.xy)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    idx = rbffd.rbffd_stencils(xy, n)
    w, st = rbffd.rbffd_weights(xy, idx, m)
    A = rbffd.rbffd_assemble(idx, w, mask, want_f32=True)
    b = rbffd.rbffd_rhs(T(f), T(g), mask)
    mg = rbffd.Multigrid(xy, mask, A)
    x, info = rbffd.rbffd_solve(A, b, opts=rbffd.make_opts(tol=1e-10, precision="mixed", mg=mg))
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10 and info["iters"] <= 40
    u = x.cpu().numpy()
    bh = oracle.rhs(f, g, d.is_dirichlet)
    rng = np.random.default_rng(11)
    rows = rng.choice(np.flatnonzero(d.is_dirichlet == 0), 200, replace=False)
    idx_o = oracle.knn_query(d.xy, n, rows)
    full = np.zeros((d.N, n), dtype=np.int32)
    full[rows] = idx_o
    w_o, _ = oracle.weights(d.xy, full, m, nodes=rows)
    uu = u[idx_o.astype(np.int64)]
    r = bh[rows] - (w_o * uu).sum(axis=1)
    bound = 1e-10 * np.linalg.norm(bh) + 1e-9 * np.abs(w_o).max(axis=1) * np.abs(uu).sum(axis=1)
    assert (np.abs(r) <= bound).all()
    # and the discrete solution approximates sin(pi x) sin(pi y) to the scheme's accuracy
    assert np.abs(u - u_ex).max() <= 1e-6
