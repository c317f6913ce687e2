"""GPU tests of the adjoint hierarchy with Galerkin coarse operators.

Each coarse operator must be the sparse triple product R A P of the level
above it (computed here on the host with scipy from the same level's arrays,
R = P^T and P_adj = (N_c / N_f) P without the coarse Dirichlet columns, both
taken from the forward hierarchy), with identity rows at coarse Dirichlet
nodes: same pattern, values to rounding.  The product is deterministic.  The
adjoint solve it right-preconditions must match the oracle's adjoint to 1e-8.
"""

import ctypes

import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from fixtures import disk_nodes, manufactured

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _gpu_system(h, m, n, seed=2107):
    from paper_2107_03632_gb300 import rbffd

    d = disk_nodes(h, seed)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    idx = rbffd.rbffd_stencils(xy, n)
    w, _ = rbffd.rbffd_weights(xy, idx, m)
    A = rbffd.rbffd_assemble(idx, w, mask, want_f32=True)
    return d, xy, mask, A


def _csr(A, n_rows, n_cols):
    return sp.csr_matrix((A.val.cpu().numpy(), A.col.cpu().numpy(), A.row_ptr.cpu().numpy()),
                         shape=(n_rows, n_cols))


def _ell(idx, val, n_cols):
    n, k = idx.shape
    return sp.csr_matrix((val.reshape(-1), idx.reshape(-1).astype(np.int64), np.arange(0, n * k + 1, k)),
                         shape=(n, n_cols))


@pytest.mark.parametrize("h,m,n", [(0.008, 4, 30), (0.012, 6, 56), (0.01, 2, 12)])
def test_galerkin_coarse_operators_are_triple_products(lib, h, m, n):
    from paper_2107_03632_gb300 import rbffd

    d, xy, mask, A = _gpu_system(h, m, n)
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    fwd = rbffd.Multigrid(xy, mask, A)
    gal = rbffd.Multigrid.galerkin_adjoint_of(fwd, AT)
    sizes = gal.levels()
    assert sizes == fwd.levels() and len(sizes) >= 3
    for l in range(len(sizes) - 1):
        Nf, Nc = sizes[l], sizes[l + 1]
        F, G, Gc = fwd.level(l), gal.level(l), gal.level(l + 1)
        cmask = Gc["is_dirichlet"].cpu().numpy().astype(bool)
        P = F["p_val"].cpu().numpy()
        pidx = F["p_idx"].cpu().numpy()
        # transfers: the prolongation (N_c / N_f) P without coarse Dirichlet columns
        p_adj = np.where(cmask[pidx], 0.0, (float(Nc) / float(Nf)) * P)
        assert np.array_equal(G["p_val"].cpu().numpy(), p_adj)
        R = _ell(pidx, P, Nc).T.tocsr()
        Pa = _ell(pidx, p_adj, Nc)
        R.eliminate_zeros()
        Pa.eliminate_zeros()
        Al = _csr(G["A"], Nf, Nf)
        keep = sp.diags((~cmask).astype(np.float64))
        eye_b = sp.diags(cmask.astype(np.float64))
        ref = (keep @ (R @ Al @ Pa) + eye_b).tocsr()
        # the structural product (all-ones values: no cancellation)
        ones = lambda M: sp.csr_matrix((np.ones_like(M.data), M.indices, M.indptr), shape=M.shape)
        pat = (keep @ (ones(R) @ ones(Al) @ ones(Pa)) + eye_b).tocsr()
        pat.sort_indices()
        got = _csr(Gc["A"], Nc, Nc)
        # the pattern: sorted columns, the structural product
        assert np.array_equal(got.indptr, pat.indptr), l
        assert np.array_equal(got.indices, pat.indices), l
        # values: to rounding of sums of ~1e3 terms per entry
        scale = abs(ref).max(axis=1).toarray().ravel()
        diff = abs(got - ref).max(axis=1).toarray().ravel()
        err = (diff / scale).max()
        assert err <= 1e-12, (l, err)
        # smoother weights from the product's own diagonal
        diag = got.diagonal()
        wref = np.where(cmask, 1.0 / diag, 0.6 / diag)
        assert np.allclose(Gc["w"].cpu().numpy(), wref, rtol=1e-15, atol=0.0)
    # coarsest: the inverse of its operator
    Lc = gal.level(len(sizes) - 1)
    Ac = _csr(Lc["A"], sizes[-1], sizes[-1]).toarray()
    assert np.abs(Lc["minv"].cpu().numpy() @ Ac - np.eye(sizes[-1])).max() <= 1e-9


def test_galerkin_product_is_deterministic(lib):
    from paper_2107_03632_gb300 import rbffd

    d, xy, mask, A = _gpu_system(0.008, 4, 30)
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    fwd = rbffd.Multigrid(xy, mask, A)
    g1 = rbffd.Multigrid.galerkin_adjoint_of(fwd, AT)
    g2 = rbffd.Multigrid.galerkin_adjoint_of(fwd, AT)
    for l in range(1, len(g1.levels())):
        a, b = g1.level(l)["A"], g2.level(l)["A"]
        for k in ("row_ptr", "col", "val"):
            assert torch.equal(getattr(a, k), getattr(b, k)), (l, k)
    r = T(np.random.default_rng(3).standard_normal(d.N))
    for fp32 in (False, True):
        assert torch.equal(g1.apply(r, fp32=fp32), g2.apply(r, fp32=fp32))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("h,m,n", [(0.03, 4, 30), (0.04, 6, 56), (0.02, 2, 12)])
def test_galerkin_adjoint_vs_oracle(lib, h, m, n, precision):
    """lambda and the gradients against the oracle's adjoint (a direct solve
    with A^T), right-preconditioned by the Galerkin hierarchy."""
    from paper_2107_03632_gb300 import rbffd

    d = disk_nodes(h)
    idx = oracle.knn(d.xy, n)
    w, _ = oracle.weights(d.xy, idx, m)
    rp, col, val = oracle.assemble(idx, w, d.is_dirichlet)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    A = rbffd.rbffd_assemble(T(idx), T(w), mask, want_f32=True)
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    fwd = rbffd.Multigrid(xy, mask, A)
    gal = rbffd.Multigrid.galerkin_adjoint_of(fwd, AT)
    rng = np.random.default_rng(5)
    dLdu = rng.standard_normal(d.N) * (d.is_dirichlet == 0)
    lam, dLdf, dLdg, info = rbffd.rbffd_solve_adjoint(AT, mask, T(dLdu),
                                                      opts=rbffd.make_opts(tol=1e-10, precision=precision, mg=gal))
    gf, gg, lam_ref = oracle.adjoint_gradient(rp, col, val, d.is_dirichlet, dLdu)
    assert info["status"] == 0 and info["iters"] <= 25, info
    scale = np.abs(lam_ref).max()
    assert np.abs(lam.cpu().numpy() - lam_ref).max() <= 1e-8 * scale
    assert np.abs(dLdf.cpu().numpy() - gf).max() <= 1e-8 * scale
    assert np.abs(dLdg.cpu().numpy() - gg).max() <= 1e-8 * scale


def test_galerkin_hierarchy_is_adjoint_only(lib):
    """A Galerkin hierarchy serves rbffd_solve_adjoint, not rbffd_solve; it
    needs a built forward hierarchy."""
    from paper_2107_03632_gb300 import rbffd

    d, xy, mask, A = _gpu_system(0.05, 2, 12)
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    fwd = rbffd.Multigrid(xy, mask, A)
    gal = rbffd.Multigrid.galerkin_adjoint_of(fwd, AT)
    b = T(np.random.default_rng(1).standard_normal(d.N))
    _, info = rbffd.rbffd_solve(A, b, opts=rbffd.make_opts(mg=gal), raise_on_error=False)
    assert info["status_code"] == 1
    lib_ = rbffd.load()
    assert lib_.rbffd_mg_galerkin_workspace_size(ctypes.byref(gal.handle)) == 0  # not a forward hierarchy


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_galerkin_adjoint_at_1M(lib, precision):
    """The misfit adjoint at ~1e6 nodes (m = 4, n = 30): right-preconditioned
    by the Galerkin hierarchy it converges to 1e-10 in at most 20 iterations;
    A^T lambda = dL/du checked in FP64 on the host."""
    from fixtures import fourier_sources
    from paper_2107_03632_gb300 import rbffd

    d, xy, mask, A = _gpu_system(1.7725e-3, 4, 30)
    _, f, g = manufactured(d.xy)
    fs = fourier_sources(d.xy, 1, 2108)[0]
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    mg = rbffd.Multigrid(xy, mask, A)
    gal = rbffd.Multigrid.galerkin_adjoint_of(mg, AT)
    o = rbffd.make_opts(tol=1e-10, precision=precision, mg=mg)
    u, _ = rbffd.rbffd_solve(A, rbffd.rbffd_rhs(T(f), T(g), mask), opts=o)
    us, _ = rbffd.rbffd_solve(A, rbffd.rbffd_rhs(T(fs), T(g), mask), opts=o)
    dLdu = rbffd.rbffd_misfit_grad(u, us, mask)
    lam, _, _, ia = rbffd.rbffd_solve_adjoint(AT, mask, dLdu, None,
                                              rbffd.make_opts(tol=1e-10, precision=precision, mg=gal))
    print(f"Galerkin adjoint at {d.N} nodes ({precision}): {ia['iters']} iterations, {ia['outer_sweeps']} passes")
    assert ia["status"] == 0 and ia["iters"] <= 20, ia
    ATs = _csr(AT, d.N, d.N)
    lam_h, g_h = lam.cpu().numpy(), dLdu.cpu().numpy()
    assert np.linalg.norm(g_h - ATs @ lam_h) <= 1e-10 * np.linalg.norm(g_h) * 1.01


def _refined_disk(h, factor, centre=(0.2, 0.1), radius=0.3, seed=2107):
    """A disk with a patch `factor` times denser: the disk's nodes outside the
    patch and, inside it, the interior nodes of a disk of spacing h / sqrt(factor)."""
    from fixtures.disk import DiskNodes

    coarse = disk_nodes(h, seed)
    fine = disk_nodes(h / np.sqrt(factor), seed + 1)
    cx, cy = centre
    out = np.hypot(coarse.xy[:, 0] - cx, coarse.xy[:, 1] - cy) >= radius
    inn = (np.hypot(fine.xy[:, 0] - cx, fine.xy[:, 1] - cy) < radius) & (fine.is_dirichlet == 0)
    interior = np.concatenate([coarse.xy[out & (coarse.is_dirichlet == 0)], fine.xy[inn]])
    boundary = coarse.xy[coarse.is_dirichlet == 1]
    xy = np.ascontiguousarray(np.concatenate([interior, boundary]))
    mask = np.zeros(xy.shape[0], dtype=np.uint8)
    mask[interior.shape[0]:] = 1
    return DiskNodes(xy, mask, float(h), int(seed), int(interior.shape[0]), int(boundary.shape[0]))


def test_galerkin_wide_rows_take_the_large_tables(lib):
    """A patch twelve times denser than the rest (radius 0.2): on the first
    level, rows of R A reach more than 512 distinct fine columns (counted here
    with scipy; ~800), more than the small hash table holds, so the level is
    redone with the large tables; the coarse operator is still the exact
    triple product."""
    from paper_2107_03632_gb300 import rbffd

    d = _refined_disk(0.01, 12.0, radius=0.2)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    idx = rbffd.rbffd_stencils(xy, 30)
    w, st = rbffd.rbffd_weights(xy, idx, 4)
    assert int(st.sum()) == 0
    A = rbffd.rbffd_assemble(idx, w, mask, want_f32=True)
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    fwd = rbffd.Multigrid(xy, mask, A)
    gal = rbffd.Multigrid.galerkin_adjoint_of(fwd, AT)
    sizes = gal.levels()
    Nf, Nc = sizes[0], sizes[1]
    F, G, Gc = fwd.level(0), gal.level(0), gal.level(1)
    cmask = Gc["is_dirichlet"].cpu().numpy().astype(bool)
    P = F["p_val"].cpu().numpy()
    pidx = F["p_idx"].cpu().numpy()
    p_adj = np.where(cmask[pidx], 0.0, (float(Nc) / float(Nf)) * P)
    R = _ell(pidx, P, Nc).T.tocsr()
    Pa = _ell(pidx, p_adj, Nc)
    R.eliminate_zeros()
    Pa.eliminate_zeros()
    Al = _csr(G["A"], Nf, Nf)
    ones = lambda M: sp.csr_matrix((np.ones_like(M.data), M.indices, M.indptr), shape=M.shape)
    RA = (ones(R) @ ones(Al)).tocsr()
    widest = int(np.diff(RA.indptr)[~cmask].max())
    assert widest > 512, widest  # the small table cannot hold these rows
    keep = sp.diags((~cmask).astype(np.float64))
    eye_b = sp.diags(cmask.astype(np.float64))
    ref = (keep @ (R @ Al @ Pa) + eye_b).tocsr()
    pat = (keep @ (RA @ ones(Pa)) + eye_b).tocsr()
    pat.sort_indices()
    got = _csr(Gc["A"], Nc, Nc)
    assert np.array_equal(got.indptr, pat.indptr) and np.array_equal(got.indices, pat.indices)
    scale = abs(ref).max(axis=1).toarray().ravel()
    assert (abs(got - ref).max(axis=1).toarray().ravel() / scale).max() <= 1e-12
    # and the adjoint it preconditions converges
    rng = np.random.default_rng(9)
    dLdu = T(rng.standard_normal(d.N) * (d.is_dirichlet == 0))
    lam, _, _, info = rbffd.rbffd_solve_adjoint(AT, mask, dLdu, opts=rbffd.make_opts(tol=1e-10, mg=gal))
    assert info["status"] == 0, info
    r = dLdu.cpu().numpy() - _csr(AT, d.N, d.N) @ lam.cpu().numpy()
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(dLdu.cpu().numpy())
