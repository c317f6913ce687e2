"""GPU parity of the batched pipeline: every (instance, rhs) solution against
the oracle's direct solve of that instance (1e-8 relative max-norm at
relative residual 1e-10), instances of uneven size and degree."""

import ctypes

import numpy as np
import pytest
import torch

import oracle
from fixtures import disk_nodes, fourier_sources, manufactured

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _batch(specs, n_rhs, seed):
    nodes, masks, fs, gs, sizes = [], [], [], [], []
    for k, (h, m, n) in enumerate(specs):
        d = disk_nodes(h, seed=seed + k)
        F = fourier_sources(d.xy, n_rhs, seed + 100 + k).T  # N x R
        u, fman, gman = manufactured(d.xy)
        F[:, 0] = fman  # first rhs: the manufactured problem
        G = np.zeros_like(F)
        G[:, 0] = gman
        nodes.append(d.xy)
        masks.append(d.is_dirichlet)
        fs.append(F)
        gs.append(G)
        sizes.append((d.N, m, n))
    return sizes, np.concatenate(nodes), np.concatenate(masks), np.concatenate(fs), np.concatenate(gs)


# (precond, persistent, device_loop): the Jacobi mixed solver; per-instance
# multigrid with one launch per (level, operation), host-driven iterations;
# the same with the persistent coarse-level kernel; with the device-side
# loop; with both.
MODES = {"jacobi": (0, 0, 0), "mg": (1, 0, 0), "mg-persistent": (1, 1, 0), "mg-device-loop": (1, 0, 1),
         "mg-persistent-device-loop": (1, 1, 1)}


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("n_rhs", [1, 2, 3, 64])
def test_batched_vs_oracle(lib, n_rhs, mode):
    """Every solver mode against the oracle's direct solves, per (instance, rhs)."""
    from paper_2107_03632_gb300 import rbffd

    specs = [(0.06, 2, 12), (0.1, 6, 56), (0.07, 4, 30), (0.09, 2, 12), (0.08, 4, 30)]
    if n_rhs == 64:
        specs = specs[:3]
    sizes, xy, mask, F, G = _batch(specs, n_rhs, 31)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    opts = rbffd.make_opts(precision="mixed", tol=1e-10)
    opts.precond, opts.persistent, opts.device_loop = MODES[mode]  # multigrid: FP64 BiCGSTAB per pair
    u, infos, st = rbffd.rbffd_solve_batched(sizes, T(xy), T(mask), T(F), T(G), opts=opts)
    u = u.cpu().numpy()
    assert st == 0 and all(i["status"] == 0 for i in infos)
    off = 0
    for (N, m, n), info in zip(sizes, infos):
        sl = slice(off, off + N)
        idx = oracle.knn(xy[sl], n)
        w, _ = oracle.weights(xy[sl], idx, m)
        rp, col, val = oracle.assemble(idx, w, mask[sl])
        for k in range(n_rhs):
            b = oracle.rhs(F[sl, k], G[sl, k], mask[sl])
            ref = oracle.solve_direct(rp, col, val, b)
            err = np.abs(u[sl, k] - ref).max() / np.abs(ref).max()
            assert err <= 1e-8, (N, m, k, err)
        assert info["rel_residual"] <= 1e-10
        off += N


def test_batched_rejects_bad_descriptors(lib):
    from paper_2107_03632_gb300 import rbffd

    descs, N = rbffd.batch_descs([(100, 4, 12)])  # n < s = 15
    assert lib.rbffd_batched_workspace_size(descs, 1, 4, None) == 0
    descs, N = rbffd.batch_descs([(100, 2, 12)])
    assert lib.rbffd_batched_workspace_size(descs, 1, 65, None) == 0
    assert lib.rbffd_batched_workspace_size(descs, 1, 64, None) > 0
    mg = rbffd.make_opts(precision="mixed")
    mg.precond = 1
    assert lib.rbffd_batched_workspace_size(descs, 1, 64, ctypes.byref(mg)) > 0


def test_batched_multigrid_multilevel_vs_oracle(lib):
    """Instances large enough for 3-4 multigrid levels each (uneven sizes
    and degrees), several right-hand sides, against the oracle's direct
    solves."""
    from paper_2107_03632_gb300 import rbffd

    specs = [(0.02, 6, 56), (0.03, 2, 12), (0.025, 4, 30)]
    R = 4
    sizes, xy, mask, F, G = _batch(specs, R, 47)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    opts = rbffd.make_opts(precision="mixed", tol=1e-10)
    opts.precond = 1
    u, infos, st = rbffd.rbffd_solve_batched(sizes, T(xy), T(mask), T(F), T(G), opts=opts)
    u = u.cpu().numpy()
    assert st == 0 and all(i["status"] == 0 for i in infos)
    assert all(i["iters"] <= 60 for i in infos), infos
    off = 0
    for (N, m, n), info in zip(sizes, infos):
        sl = slice(off, off + N)
        idx = oracle.knn(xy[sl], n)
        w, _ = oracle.weights(xy[sl], idx, m)
        rp, col, val = oracle.assemble(idx, w, mask[sl])
        for k in range(R):
            b = oracle.rhs(F[sl, k], G[sl, k], mask[sl])
            ref = oracle.solve_direct(rp, col, val, b)
            err = np.abs(u[sl, k] - ref).max() / np.abs(ref).max()
            assert err <= 1e-8, (N, m, k, err)
        assert info["rel_residual"] <= 1e-10
        off += N


@pytest.mark.parametrize("device_loop", [0, 1])
def test_batched_bounded_wait_times_out_and_the_context_survives(lib, device_loop):
    """The persistent coarse-level kernel's waits are bounded: with its test
    hook the first task waits on a counter that nothing increments, so after
    spin_limit polls the kernel records a timeout, every block stops, and the
    solve returns RBFFD_ERR_TIMEOUT (no fault, no hang).  A normal solve on the
    same context afterwards matches the oracle."""
    from paper_2107_03632_gb300 import rbffd

    specs = [(0.03, 4, 30), (0.04, 2, 12)]  # multi-level instances (coarse tasks exist)
    sizes, xy, mask, F, G = _batch(specs, 3, 47)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    opts = rbffd.make_opts(precision="mixed", tol=1e-10)
    opts.precond = 1
    opts.persistent = 1
    opts.device_loop = device_loop
    opts.spin_limit = 2000
    opts.wait_test = 1
    _, infos, st = rbffd.rbffd_solve_batched(sizes, T(xy), T(mask), T(F), T(G), opts=opts, raise_on_error=False)
    assert st == rbffd.RBFFD_ERR_TIMEOUT
    torch.cuda.synchronize()
    opts.wait_test = 0
    opts.spin_limit = 0
    u, infos, st = rbffd.rbffd_solve_batched(sizes, T(xy), T(mask), T(F), T(G), opts=opts)
    assert st == 0 and all(i["status"] == 0 for i in infos)
    u = u.cpu().numpy()
    off = 0
    for (N, m, n) in sizes:
        sl = slice(off, off + N)
        idx = oracle.knn(xy[sl], n)
        w, _ = oracle.weights(xy[sl], idx, m)
        rp, col, val = oracle.assemble(idx, w, mask[sl])
        for k in range(3):
            ref = oracle.solve_direct(rp, col, val, oracle.rhs(F[sl, k], G[sl, k], mask[sl]))
            assert np.abs(u[sl, k] - ref).max() / np.abs(ref).max() <= 1e-8
        off += N
