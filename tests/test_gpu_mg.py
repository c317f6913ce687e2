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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("h,m,n", [(0.03, 4, 30), (0.04, 6, 56)])
def test_mg_adjoint_vs_oracle(lib, h, m, n, precision):
    """The adjoint solve A^T lambda = dL/du with the transposed hierarchy:
    lambda and the gradients match the oracle's adjoint (direct solve with
    A^T) to 1e-8, in few iterations."""
    from paper_2107_03632_gb300 import rbffd

    d, idx, w, rp, col, val, b = _system(h, m, n)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    A = rbffd.rbffd_assemble(T(idx), T(w), mask, want_f32=True)
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    rng = np.random.default_rng(5)
    dLdu = rng.standard_normal(d.N) * (d.is_dirichlet == 0)
    mga = rbffd.Multigrid(xy, mask, AT, adjoint=True)
    lam, dLdf, dLdg, info = rbffd.rbffd_solve_adjoint(AT, mask, T(dLdu),
                                                      opts=rbffd.make_opts(tol=1e-10, precision=precision, mg=mga))
    gf, gg, lam_ref = oracle.adjoint_gradient(rp, col, val, d.is_dirichlet, dLdu)
    assert info["status"] == 0 and info["iters"] <= 40, info
    scale = np.abs(lam_ref).max()
    assert np.abs(lam.cpu().numpy() - lam_ref).max() <= 1e-8 * scale
    assert np.abs(dLdf.cpu().numpy() - gf).max() <= 1e-8 * scale
    assert np.abs(dLdg.cpu().numpy() - gg).max() <= 1e-8 * scale


def test_mg_forward_and_adjoint_hierarchies_are_not_interchangeable(lib):
    from paper_2107_03632_gb300 import rbffd

    d, idx, w, rp, col, val, b = _system(0.05, 2, 12)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    A = rbffd.rbffd_assemble(T(idx), T(w), mask)
    AT = rbffd.rbffd_transpose(A)
    fwd = rbffd.Multigrid(xy, mask, A)
    adj = rbffd.Multigrid(xy, mask, AT, adjoint=True)
    _, info = rbffd.rbffd_solve(A, T(b), opts=rbffd.make_opts(mg=adj), raise_on_error=False)
    assert info["status_code"] == 1
    _, _, _, info = rbffd.rbffd_solve_adjoint(AT, mask, T(b), opts=rbffd.make_opts(mg=fwd), raise_on_error=False)
    assert info["status_code"] == 1


def test_misfit_grad_bitexact(lib):
    from paper_2107_03632_gb300 import rbffd

    rng = np.random.default_rng(9)
    N = 100003
    u, ut = rng.standard_normal(N), rng.standard_normal(N)
    mask = (rng.random(N) < 0.1).astype(np.uint8)
    g = rbffd.rbffd_misfit_grad(T(u), T(ut), T(mask)).cpu().numpy()
    assert np.array_equal(g, np.where(mask == 1, 0.0, 2.0 * (u - ut)))


def _gpu_system(h, m, n, seed=2107):
    from paper_2107_03632_gb300 import rbffd

    d = disk_nodes(h, seed)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    idx = rbffd.rbffd_stencils(xy, n)
    w, _ = rbffd.rbffd_weights(xy, idx, m)
    A = rbffd.rbffd_assemble(idx, w, mask, want_f32=True)
    return d, xy, mask, A


def _scipy(A, n):
    import scipy.sparse as sp

    return sp.csr_matrix((A.val.cpu().numpy(), A.col.cpu().numpy(), A.row_ptr.cpu().numpy()), shape=(n, n))


def test_mg_level_views_and_transposed_hierarchy(lib):
    """Level views: level 0 is the caller's operator; every coarse node is a
    fine node; the smoother weights are omega / a_ii inside and 1 / a_ii on
    Dirichlet rows; the coarsest level carries the inverse of its operator.
    The adjoint hierarchy holds the transposes of the forward operators and
    R^T = (N_c / N_f) P without the coarse Dirichlet columns as prolongation."""
    from paper_2107_03632_gb300 import rbffd

    d, xy, mask, A = _gpu_system(0.01, 4, 30)
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    mg = rbffd.Multigrid(xy, mask, A, omega=0.6)
    mga = rbffd.Multigrid(xy, mask, AT, omega=0.6, adjoint=True)
    sizes = mg.levels()
    assert sizes == mga.levels() and len(sizes) >= 3
    prev = None
    for l, n in enumerate(sizes):
        f, a = mg.level(l), mga.level(l)
        assert f["n_nodes"] == n
        Af, Aa = _scipy(f["A"], n), _scipy(a["A"], n)
        if l == 0:
            assert (Af != _scipy(A, n)).nnz == 0
        # the adjoint's operator is the forward one transposed, bit for bit
        assert (Af.T.tocsr() != Aa).nnz == 0
        m = f["is_dirichlet"].cpu().numpy().astype(bool)
        diag = Af.diagonal()
        want = np.where(m, 1.0, 0.6) / diag
        assert np.allclose(f["w"].cpu().numpy(), want, rtol=1e-15, atol=0)
        assert np.all(diag[m] == 1.0)
        if prev is not None:
            # coarse nodes are a subset of the finer level's nodes
            fine = {tuple(p) for p in prev["xy"].cpu().numpy()}
            assert all(tuple(p) in fine for p in f["xy"].cpu().numpy())
            # prolongation into the finer level: adjoint = scaled forward,
            # coarse Dirichlet columns zeroed
            pv, av = prev["fwd_p_val"], prev["adj_p_val"]
            pidx = prev["p_idx"]
            scale = n / prev["n_nodes"]
            cm = m[pidx]
            assert np.array_equal(av, np.where(cm, 0.0, pv * scale))
            # the interpolation reproduces quadratics at every interior fine
            # node (PHS r^3 + degree-2 weights), rows of Dirichlet nodes are 0
            fxy, cxy = prev["xy"].cpu().numpy(), f["xy"].cpu().numpy()
            fm = prev["mask"]
            assert np.all(pv[fm] == 0.0)
            nb = cxy[pidx]  # fine x 12 x 2
            for px, py in ((0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)):
                got = (pv * nb[..., 0] ** px * nb[..., 1] ** py).sum(axis=1)
                want = fxy[:, 0] ** px * fxy[:, 1] ** py
                err = np.abs(got - want)[~fm]
                # (rows of singular interpolation systems fall back to the
                # nearest coarse node: constants only)
                assert np.quantile(err, 0.999) <= 1e-10, (l, px, py, np.quantile(err, 0.999))
                if px == py == 0:
                    assert err.max() <= 1e-12
        if l == len(sizes) - 1:
            assert f["p_idx"] is None and f["minv"] is not None
            Ad = Af.toarray()
            assert np.abs(f["minv"].cpu().numpy() @ Ad - np.eye(n)).max() <= 1e-10
        else:
            assert f["minv"] is None
            assert torch.equal(f["p_idx"], a["p_idx"])
        prev = {"xy": f["xy"], "n_nodes": n, "mask": m,
                "p_idx": None if f["p_idx"] is None else f["p_idx"].cpu().numpy(),
                "fwd_p_val": None if f["p_val"] is None else f["p_val"].cpu().numpy(),
                "adj_p_val": None if a["p_val"] is None else a["p_val"].cpu().numpy()}


@pytest.mark.parametrize("fp32", [False, True])
def test_mg_adjoint_cycle_is_exact_transpose(lib, fp32):
    """The adjoint preconditioner is the transpose of the forward one on the
    residuals a forward solve produces (zero on Dirichlet rows):
    r . (B s) == (M^T r) . s for every r and every s with s_b = 0, and it maps
    Dirichlet entries as the back substitution x_b = r_b - sum_i a_ib x_i."""
    from paper_2107_03632_gb300 import rbffd

    d, xy, mask, A = _gpu_system(0.006, 6, 56)
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    mg = rbffd.Multigrid(xy, mask, A)
    mga = rbffd.Multigrid(xy, mask, AT, adjoint=True)
    rng = np.random.default_rng(5)
    m = d.is_dirichlet.astype(bool)
    for _ in range(3):
        r = rng.standard_normal(d.N)
        s = np.where(m, 0.0, rng.standard_normal(d.N))
        Bs = mg.apply(T(s), fp32=fp32).cpu().numpy()
        Mr = mga.apply(T(r), fp32=fp32).cpu().numpy()
        lhs, rhs = r @ Bs, Mr @ s
        tol = 1e-5 if fp32 else 1e-12
        assert abs(lhs - rhs) <= tol * np.linalg.norm(r) * np.linalg.norm(Bs), (lhs, rhs)
        assert np.all(Bs[m] == 0.0)  # boundary-free in, boundary-free out
        # Dirichlet entries of M^T r: the back substitution
        ATs = _scipy(AT, d.N)
        resid = r - ATs @ Mr
        assert np.abs(resid[m]).max() <= 1e-12 * np.abs(r).max() * 100


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mg_boundary_data_and_adjoint_at_1M(lib, precision):
    """Right-hand sides with boundary data (a Fourier source with the
    manufactured boundary values) and the adjoint of a misfit at ~1e6 nodes:
    both converge to 1e-10 within a few dozen iterations."""
    from fixtures import fourier_sources
    from paper_2107_03632_gb300 import rbffd

    d, xy, mask, A = _gpu_system(1.7725e-3, 4, 30)
    _, f, g = manufactured(d.xy)
    fs = fourier_sources(d.xy, 1, 2108)[0]
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    mg = rbffd.Multigrid(xy, mask, A)
    mga = rbffd.Multigrid(xy, mask, AT, adjoint=True)
    o = rbffd.make_opts(tol=1e-10, precision=precision, mg=mg)
    u, i1 = rbffd.rbffd_solve(A, rbffd.rbffd_rhs(T(f), T(g), mask), opts=o)
    us, i2 = rbffd.rbffd_solve(A, rbffd.rbffd_rhs(T(fs), T(g), mask), opts=o)
    for info in (i1, i2):
        assert info["status"] == 0 and info["iters"] <= 30, info
    dLdu = rbffd.rbffd_misfit_grad(u, us, mask)
    lam, dLdf, dLdg, ia = rbffd.rbffd_solve_adjoint(AT, mask, dLdu, None,
                                                   rbffd.make_opts(tol=1e-10, precision=precision, mg=mga))
    # the adjoint runs left preconditioned: robust, but its preconditioned
    # residual hides rough residual components by ~h^2, so it takes two or
    # three passes (~13 iterations each)
    assert ia["status"] == 0 and ia["iters"] <= 60, ia
    # check A^T lambda = dL/du in FP64 on the host
    ATs = _scipy(AT, d.N)
    lam_h, g_h = lam.cpu().numpy(), dLdu.cpu().numpy()
    assert np.linalg.norm(g_h - ATs @ lam_h) <= 1e-10 * np.linalg.norm(g_h) * 1.01


def test_mg_adjoint_of_forward_equals_adjoint_setup(lib):
    """rbffd_mg_adjoint_of (coarse levels reused from the forward hierarchy)
    holds the same values as rbffd_mg_setup_adjoint, bit for bit, and applies
    the same preconditioner."""
    from paper_2107_03632_gb300 import rbffd

    d, xy, mask, A = _gpu_system(0.008, 4, 30)
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    mg = rbffd.Multigrid(xy, mask, A)
    m1 = rbffd.Multigrid(xy, mask, AT, adjoint=True)
    m2 = rbffd.Multigrid.adjoint_of(mg, AT)
    assert m1.levels() == m2.levels()
    for l in range(len(m1.levels())):
        a, b = m1.level(l), m2.level(l)
        for k in ("xy", "is_dirichlet", "w", "p_idx", "p_val", "minv"):
            assert (a[k] is None) == (b[k] is None), k
            if a[k] is not None:
                assert torch.equal(a[k], b[k]), (l, k)
        for k in ("row_ptr", "col", "val"):
            assert torch.equal(getattr(a["A"], k), getattr(b["A"], k)), (l, k)
    r = T(np.random.default_rng(2).standard_normal(d.N))
    for fp32 in (False, True):
        assert torch.equal(m1.apply(r, fp32=fp32), m2.apply(r, fp32=fp32))
    # the forward hierarchy may be rebuilt afterwards: m2 owns its arrays
    mg.setup(xy, mask, A)
    assert torch.equal(m1.apply(r), m2.apply(r))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("use_mg", [True, False])
def test_solver_stops_on_stagnation(lib, precision, use_mg):
    """Unisolvent stencils (m = 4, n = s = 15) give an operator with spurious
    modes on which BiCGSTAB stalls: the solve must give up early
    (RBFFD_ERR_NOT_CONVERGED after a few thousand iterations, not max_iter),
    and report the residual it reached."""
    from paper_2107_03632_gb300 import rbffd

    d, xy, mask, A = _gpu_system(0.01, 4, 15)
    _, f, g = manufactured(d.xy)
    b = rbffd.rbffd_rhs(T(f), T(g), mask)
    mg = rbffd.Multigrid(xy, mask, A) if use_mg else None
    x, info = rbffd.rbffd_solve(A, b, opts=rbffd.make_opts(tol=1e-10, precision=precision, mg=mg, max_iter=200000),
                                raise_on_error=False)
    assert info["status_code"] == 4, info
    assert info["iters"] <= 5000, info
    assert np.isfinite(info["rel_residual"]) and info["rel_residual"] > 1e-10


@pytest.mark.parametrize("h,m,n", [(0.02, 4, 30), (0.1, 2, 12)])
def test_two_phase_setup_equals_one_call(lib, h, m, n):
    """rbffd_mg_setup_geometry on a second stream while the fine weights are
    computed, then rbffd_mg_setup_operator: the same hierarchy as
    rbffd_mg_setup (identical levels, V-cycle outputs and solutions, bit for
    bit).  h = 0.1: a node set that is a single (dense) level."""
    from paper_2107_03632_gb300 import rbffd

    d, idx, w, rp, col, val, b = _system(h, m, n)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    idx_t = T(idx)
    w1, _ = rbffd.rbffd_weights(xy, idx_t, m)
    A = rbffd.rbffd_assemble(idx_t, w1, mask, want_f32=True)
    one = rbffd.Multigrid(xy, mask, A)
    # the second hierarchy: the same weights again on the current stream (the
    # same bits), the geometry on a side stream meanwhile
    side = torch.cuda.Stream(DEV)
    two = rbffd.Multigrid(xy, mask, A, ws=torch.empty_like(one.ws))
    w2, _ = rbffd.rbffd_weights(xy, idx_t, m)  # in flight while the geometry is built
    two.setup_geometry(xy, mask, stream=side)
    A2 = rbffd.rbffd_assemble(idx_t, w2, mask, want_f32=True)
    two.setup_operator(A2)
    assert torch.equal(A2.val, A.val)
    assert two.levels() == one.levels()
    for l in range(len(one.levels())):
        a, c = one.level(l), two.level(l)
        for k in ("xy", "is_dirichlet", "w", "p_idx", "p_val", "minv"):
            if a.get(k) is not None:
                assert torch.equal(a[k], c[k]), (l, k)
        if l > 0:
            assert torch.equal(a["A"].val, c["A"].val) and torch.equal(a["A"].col, c["A"].col)
    bb = T(b)
    for fp32 in (False, True):
        assert torch.equal(one.apply(bb, fp32=fp32), two.apply(bb, fp32=fp32))
    for prec in ("fp64", "mixed"):
        x1, i1 = rbffd.rbffd_solve(A, bb, opts=rbffd.make_opts(precision=prec, mg=one))
        x2, i2 = rbffd.rbffd_solve(A2, bb, opts=rbffd.make_opts(precision=prec, mg=two))
        assert torch.equal(x1, x2) and i1["iters"] == i2["iters"], prec


def test_two_phase_setup_refuses_misuse(lib):
    """A hierarchy between the two phases serves no solve; the operator phase
    takes only a geometry of the same node count."""
    from paper_2107_03632_gb300 import rbffd

    d, idx, w, rp, col, val, b = _system(0.04, 2, 12)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    A = rbffd.rbffd_assemble(T(idx), T(w), mask, want_f32=True)
    mg = rbffd.Multigrid(xy, mask, A)
    mg.setup_geometry(xy, mask)
    x, info = rbffd.rbffd_solve(A, T(b), opts=rbffd.make_opts(mg=mg), raise_on_error=False)
    assert info["status_code"] == 1  # RBFFD_ERR_INVALID_ARG
    d2, idx2, w2, *_ = _system(0.05, 2, 12)
    A_other = rbffd.rbffd_assemble(T(idx2), T(w2), T(d2.is_dirichlet), want_f32=True)
    with pytest.raises(rbffd.RbffdError):
        mg.setup_operator(A_other)
    mg.setup_operator(A)
    with pytest.raises(rbffd.RbffdError):
        mg.setup_operator(A)  # already attached
    x, info = rbffd.rbffd_solve(A, T(b), opts=rbffd.make_opts(mg=mg))
    assert info["status"] == 0
