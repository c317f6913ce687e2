"""Pins of the CPU oracle to the paper and to mathematics (no GPU).

Each test ties one oracle function to something other than itself: values
worked by hand or printed in the paper (tests/golden/), closed forms,
invariants, special cases that reduce to textbook results, an independent
library routine, or an extended-precision re-solve.
"""

import math
import os

import mpmath
import numpy as np
import pytest
import scipy.linalg
import scipy.spatial

import oracle
from conftest import ROOT
from fixtures import disk_nodes, manufactured, splitmix64, uniform01
from oracle.assemble import to_scipy

GOLDEN = os.path.join(ROOT, "tests", "golden")


def golden_rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


# ------------------------------------------------------------------- knn -----
def test_knn_hand_worked_line():
    rows = golden_rows("knn_line.txt")
    nodes = [r for r in rows if r[0] != "STENCIL"]
    xy = np.array([[float(r[1]), 0.0] for r in nodes])
    want = {int(r[1]): [int(v) for v in r[2:]] for r in rows if r[0] == "STENCIL"}
    idx = oracle.knn(xy, 4)
    for i, s in want.items():
        assert list(idx[i]) == s


def test_knn_matches_kdtree_on_jittered_disk():
    """Against scipy's k-d tree.  Where the tree's distances are separated by
    more than rounding the order is unique and must match exactly; the
    equispaced boundary nodes give near-ties (mirror-image neighbours), where
    only the distances themselves must agree."""
    d = disk_nodes(0.04)
    for n in (12, 30, 56):
        idx = oracle.knn(d.xy, n)
        dist, ref = scipy.spatial.cKDTree(d.xy).query(d.xy, k=n + 1)
        gaps = np.diff(dist, axis=1)
        clear = (gaps > 1e-12 * dist[:, -1:]).all(axis=1)
        assert clear.mean() > 0.9
        assert np.array_equal(idx[clear], ref[clear, :n])
        mine = np.sqrt(((d.xy[idx] - d.xy[:, None, :]) ** 2).sum(axis=2))
        np.testing.assert_allclose(mine, dist[:, :n], rtol=1e-12, atol=1e-15)
        assert np.all(idx[:, 0] == np.arange(d.N))  # each node leads its own stencil


def test_knn_exact_grid_ties_broken_by_index():
    """h = 1/16 makes grid coordinates and their differences exact, so the
    four axis neighbours tie exactly and must appear in index order."""
    d = disk_nodes(1.0 / 16.0, jitter=0.0)
    idx = oracle.knn(d.xy, 9)
    xy = d.xy
    interior = np.nonzero((d.is_dirichlet == 0) & (np.hypot(xy[:, 0], xy[:, 1]) < 0.5))[0]
    for i in interior[:50]:
        s = idx[i]
        assert s[0] == i
        d2 = ((xy[s] - xy[i]) ** 2).sum(axis=1)
        assert np.all(d2[1:5] == 1.0 / 256.0) and np.all(d2[5:9] == 2.0 / 256.0)
        assert list(s[1:5]) == sorted(s[1:5]) and list(s[5:9]) == sorted(s[5:9])


def test_knn_query_sample_equals_full():
    d = disk_nodes(0.05)
    q = np.array([0, 7, 100, d.N - 1])
    assert np.array_equal(oracle.knn_query(d.xy, 20, q), oracle.knn(d.xy, 20)[q])


# --------------------------------------------------------------- weights -----
def test_weights_five_point_special_case():
    rows = golden_rows("five_point_laplacian.txt")
    pts = np.array([[float(a), float(b)] for a, b in rows[:6]])
    want = np.array([float(v) for v in rows[6]])
    for h in (1.0, 0.01, 3.7e-4):
        xy = pts * h
        w, st = oracle.weights(xy, np.arange(6)[None, :], 2, nodes=np.array([0]))
        assert st[0] == 0
        np.testing.assert_allclose(w[0] * h * h, want, rtol=0, atol=1e-11)


def _random_stencils(m, n, count, seed):
    d = disk_nodes(0.05, seed=seed)
    idx = oracle.knn(d.xy, n)
    nodes = np.arange(0, d.N, max(1, d.N // count))[:count]
    return d, idx, nodes


@pytest.mark.parametrize("m,n", [(2, 12), (4, 30), (6, 56), (2, 30), (4, 45)])
def test_weights_reproduce_laplacian_of_monomials(m, n):
    """P^T w = lap p exactly for every monomial of degree <= m, incl. sum(w) = 0."""
    d, idx, nodes = _random_stencils(m, n, 40, 11)
    w, st = oracle.weights(d.xy, idx, m, nodes=nodes)
    assert not st.any()
    for r, i in enumerate(nodes):
        X = d.xy[idx[i]] - d.xy[i]
        for a in range(m + 1):
            for b in range(m + 1 - a):
                p = X[:, 0] ** a * X[:, 1] ** b
                want = 2.0 if (a, b) in ((2, 0), (0, 2)) else 0.0
                scale = np.abs(w[r] * p).sum() + abs(want)
                assert abs((w[r] * p).sum() - want) <= 1e-9 * scale


def _interp_laplacian(stencil_xy, centre, u_vals, m):
    """Laplacian at `centre` of the PHS r^3 + degree-m interpolant of u_vals,
    built independently of the oracle (cdist, explicit monomials, scipy
    solve) and differentiated numerically (fourth-order central differences
    with Richardson extrapolation), so no analytic lap r^3 is used."""
    n = stencil_xy.shape[0]
    ex = [(dd - i, i) for dd in range(m + 1) for i in range(dd + 1)]
    D = scipy.spatial.distance.cdist(stencil_xy, stencil_xy)
    P = np.array([[x ** a * y ** b for (a, b) in ex] for x, y in stencil_xy])
    s = P.shape[1]
    K = np.zeros((n + s, n + s))
    K[:n, :n] = D ** 3
    K[:n, n:] = P
    K[n:, :n] = P.T
    coef = scipy.linalg.solve(K, np.concatenate([u_vals, np.zeros(s)]))
    c, dcoef = coef[:n], coef[n:]

    # |x - x_c|^3 is only C^2 at x_c, which would leave an O(eps) finite-
    # difference error; its Laplacian there is 0 (the limit of any multiple
    # of r), so that one term is left out and the smooth rest differentiated.
    smooth = np.hypot(*(stencil_xy - centre).T) > 0

    def s_eval(pt):
        r = np.hypot(stencil_xy[:, 0] - pt[0], stencil_xy[:, 1] - pt[1])
        return (c[smooth] * r[smooth] ** 3).sum() + sum(dc * pt[0] ** a * pt[1] ** b
                                                        for dc, (a, b) in zip(dcoef, ex))

    def fd(eps):
        tot = 0.0
        for e in (np.array([eps, 0.0]), np.array([0.0, eps])):
            f2 = s_eval(centre + 2 * e) + s_eval(centre - 2 * e)
            f1 = s_eval(centre + e) + s_eval(centre - e)
            tot += (-f2 + 16 * f1 - 30 * s_eval(centre)) / (12 * eps * eps)
        return tot

    h = 1e-3 * np.abs(stencil_xy - centre).max()
    return (16 * fd(h / 2) - fd(h)) / 15


@pytest.mark.parametrize("m,n", [(2, 12), (4, 30), (2, 20)])
def test_weights_apply_laplacian_of_rbf_interpolant(m, n):
    """sum_j w_j u_j equals lap of the PHS+poly interpolant of u at x_c; this
    pins the radial part of the system (the 9 r right-hand side, the r^3
    kernel, the scaling), which polynomial reproduction cannot see."""
    d, idx, nodes = _random_stencils(m, n, 6, 21)
    w, _ = oracle.weights(d.xy, idx, m, nodes=nodes)
    rng = np.random.default_rng(1)
    for r, i in enumerate(nodes):
        sx = d.xy[idx[i]]
        u = np.exp(sx[:, 0]) * np.cos(2.0 * sx[:, 1]) + rng.standard_normal(n) * 0.1
        lap_interp = _interp_laplacian(sx, d.xy[i], u, m)
        assert abs((w[r] * u).sum() - lap_interp) <= 2e-5 * np.abs(w[r] * u).sum()


def test_weights_scale_and_shift_invariance():
    d, idx, nodes = _random_stencils(4, 30, 10, 3)
    w, _ = oracle.weights(d.xy, idx, 4, nodes=nodes)
    lam = 2.5
    w2, _ = oracle.weights(d.xy * lam + np.array([3.0, -7.0]), idx, 4, nodes=nodes)
    np.testing.assert_allclose(w2 * lam * lam, w, rtol=1e-9, atol=1e-9 * np.abs(w).max())


def test_weights_grid_symmetry():
    """On an exact grid the weights of mirror-image neighbours are equal."""
    d = disk_nodes(1.0 / 16.0, jitter=0.0)
    idx = oracle.knn(d.xy, 13)  # centre, 4 axis, 4 diagonal, 4 at distance 2
    c = int(np.argmin(np.hypot(d.xy[:, 0], d.xy[:, 1])))
    w, _ = oracle.weights(d.xy, idx, 2, nodes=np.array([c]))
    X = np.round((d.xy[idx[c]] - d.xy[c]) * 16).astype(int)
    wd = {tuple(p): v for p, v in zip(X, w[0])}
    for ring in ([(1, 0), (-1, 0), (0, 1), (0, -1)], [(1, 1), (-1, 1), (1, -1), (-1, -1)],
                 [(2, 0), (-2, 0), (0, 2), (0, -2)]):
        vals = [wd[p] for p in ring]
        assert max(vals) - min(vals) <= 1e-9 * max(abs(v) for v in vals)


@pytest.mark.parametrize("m,n,hs", [(2, 12, (0.1, 0.05, 0.025)), (4, 30, (0.1, 0.05, 0.025)),
                                    (6, 56, (0.2, 0.1, 0.05))])
def test_weights_consistency_order(m, n, hs):
    """The RMS of sum w u - lap u over nodes away from the boundary falls
    like h^(m-1) (degree-m reproduction of a second derivative), with 0.25
    of slack for the scatter of jittered nodes."""
    min_order = m - 1 - 0.25
    errs = []
    for h in hs:
        d = disk_nodes(h, seed=5)
        u, f, _ = manufactured(d.xy)
        far = np.nonzero(np.hypot(d.xy[:, 0], d.xy[:, 1]) < 0.5)[0]
        idx = oracle.knn(d.xy, n)
        w, _ = oracle.weights(d.xy, idx, m, nodes=far)
        approx = (w * u[idx[far]]).sum(axis=1)
        errs.append(np.sqrt(((approx + f[far]) ** 2).mean()))  # lap u = -f
    orders = [math.log(errs[k] / errs[k + 1]) / math.log(hs[k] / hs[k + 1]) for k in range(len(hs) - 1)]
    assert min(orders) >= min_order, (errs, orders)


def test_weights_fp64_error_vs_extended_precision():
    """An mpmath (40 digits) re-solve of m = 6 stencils bounds the FP64
    oracle's own rounding error well below the 1e-7 parity tolerance."""
    d, idx, nodes = _random_stencils(6, 56, 3, 9)
    w, _ = oracle.weights(d.xy, idx, 6, nodes=nodes)
    mpmath.mp.dps = 40
    for r, i in enumerate(nodes):
        X = d.xy[idx[i]] - d.xy[i]
        delta = math.sqrt(((X ** 2).sum(axis=1)).max())
        xs = [(mpmath.mpf(float(a)) / delta, mpmath.mpf(float(b)) / delta) for a, b in X]
        ex = oracle.monomial_exponents(6)
        n, s = len(xs), len(ex)
        K = mpmath.zeros(n + s, n + s)
        rhs = mpmath.zeros(n + s, 1)
        for j in range(n):
            for k in range(n):
                K[j, k] = mpmath.sqrt((xs[j][0] - xs[k][0]) ** 2 + (xs[j][1] - xs[k][1]) ** 2) ** 3
            for q, (a, b) in enumerate(ex):
                K[j, n + q] = K[n + q, j] = xs[j][0] ** a * xs[j][1] ** b
            rhs[j] = 9 * mpmath.sqrt(xs[j][0] ** 2 + xs[j][1] ** 2)
        for q, (a, b) in enumerate(ex):
            rhs[n + q] = 2 if (a, b) in ((2, 0), (0, 2)) else 0
        sol = mpmath.lu_solve(K, rhs)
        w_hp = np.array([float(sol[j]) for j in range(n)]) / (delta * delta)
        assert np.abs(w[r] - w_hp).max() / np.abs(w_hp).max() <= 1e-8


# -------------------------------------------------------------- assembly -----
def test_assembly_structure_and_consistency():
    d = disk_nodes(0.05)
    u, f, g = manufactured(d.xy)
    idx = oracle.knn(d.xy, 30)
    w, _ = oracle.weights(d.xy, idx, 4)
    rp, col, val = oracle.assemble(idx, w, d.is_dirichlet)
    nb = int(d.is_dirichlet.sum())
    assert rp[-1] == (d.N - nb) * 30 + nb
    A = to_scipy(rp, col, val, d.N)
    b = oracle.rhs(f, g, d.is_dirichlet)
    res = A @ u - b
    dm = d.is_dirichlet.astype(bool)
    assert np.all(res[dm] == 0.0)  # identity rows, g = u on the boundary
    assert np.abs(res[~dm]).max() < 1e-2 * np.abs(f).max()  # consistency error of lap u = -f
    for i in np.nonzero(dm)[0][:10]:
        assert A[i, i] == 1.0 and A.getrow(i).nnz == 1
    i = int(np.nonzero(~dm)[0][3])
    assert list(col[rp[i]:rp[i + 1]]) == list(idx[i]) and np.array_equal(val[rp[i]:rp[i + 1]], w[i])


# ----------------------------------------------------------------- solve -----
def test_direct_solve_residual_and_dense_sparse_agree():
    d = disk_nodes(0.04)
    u, f, g = manufactured(d.xy)
    uh, (idx, w, rp, col, val, b) = oracle.poisson_solve(d.xy, d.is_dirichlet, f, g, 2, 12)
    A = to_scipy(rp, col, val, d.N)
    assert np.linalg.norm(A @ uh - b) / np.linalg.norm(b) < 1e-13
    import scipy.sparse.linalg as spla

    us = spla.splu(A.tocsc()).solve(b)
    assert np.abs(us - uh).max() / np.abs(uh).max() < 1e-11


@pytest.mark.parametrize("m,n,hs", [(2, 12, (0.08, 0.04, 0.02)), (4, 30, (0.1, 0.05, 0.025)),
                                    (6, 56, (0.2, 0.1, 0.05))])
def test_solution_converges_to_manufactured_solution(m, n, hs):
    """max |u_h - sin(pi x) sin(pi y)| falls with slope >= m - 1 - 0.25."""
    errs = []
    for h in hs:
        d = disk_nodes(h)
        u, f, g = manufactured(d.xy)
        uh, _ = oracle.poisson_solve(d.xy, d.is_dirichlet, f, g, m, n)
        errs.append(np.abs(uh - u).max())
    slopes = [math.log(errs[k] / errs[k + 1]) / math.log(hs[k] / hs[k + 1]) for k in range(len(hs) - 1)]
    assert min(slopes) >= m - 1 - 0.25, (errs, slopes)


# --------------------------------------------------------------- adjoint -----
def test_adjoint_gradient_matches_central_differences():
    """L = sum_interior (u - u*)^2 is quadratic in (f, g), so central
    differences equal <grad L, v> up to rounding."""
    d = disk_nodes(0.08)
    u_ex, f, g = manufactured(d.xy)
    idx = oracle.knn(d.xy, 12)
    w, _ = oracle.weights(d.xy, idx, 2)
    rp, col, val = oracle.assemble(idx, w, d.is_dirichlet)
    dm = d.is_dirichlet.astype(bool)
    u_star = np.sin(2.0 * d.xy[:, 0] + d.xy[:, 1])

    def loss(ff, gg):
        uu = oracle.solve_direct(rp, col, val, oracle.rhs(ff, gg, d.is_dirichlet))
        return float(((uu - u_star)[~dm] ** 2).sum()), uu

    L0, u0 = loss(f, g)
    dLdu = np.where(dm, 0.0, 2.0 * (u0 - u_star))
    gf, gg, lam = oracle.adjoint_gradient(rp, col, val, d.is_dirichlet, dLdu)
    assert np.all(gf[dm] == 0.0) and np.all(gg[~dm] == 0.0)
    rng = np.random.default_rng(0)
    for _ in range(4):
        vf, vg = rng.standard_normal(d.N), rng.standard_normal(d.N)
        vf /= np.abs(vf).max()
        vg /= np.abs(vg).max()
        eps = 1e-6 * max(np.abs(f).max(), 1.0)
        Lp, _ = loss(f + eps * vf, g + eps * vg)
        Lm, _ = loss(f - eps * vf, g - eps * vg)
        fd = (Lp - Lm) / (2 * eps)
        an = gf @ vf + gg @ vg
        assert abs(fd - an) <= 1e-6 * max(abs(fd), abs(an))


def test_adjoint_duality_identity():
    """<lambda, b'> = <dL/du, A^-1 b'> for any perturbation b'."""
    d = disk_nodes(0.08)
    idx = oracle.knn(d.xy, 30)
    w, _ = oracle.weights(d.xy, idx, 4)
    rp, col, val = oracle.assemble(idx, w, d.is_dirichlet)
    rng = np.random.default_rng(4)
    dLdu, bp = rng.standard_normal(d.N), rng.standard_normal(d.N)
    _, _, lam = oracle.adjoint_gradient(rp, col, val, d.is_dirichlet, dLdu)
    lhs = lam @ bp
    rhs = dLdu @ oracle.solve_direct(rp, col, val, bp)
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1.0)


# -------------------------------------------------- explicit loop (Eq. 4) -----
def test_table1_l2_estimate_column():
    for n, est, _observed in golden_rows("table1_l2_estimate.txt"):
        assert oracle.l2_estimate_nodes(5.5e6, int(n)) == int(est)


def test_explicit_step_fixed_point_and_boundary():
    """The steady solution is a fixed point of Eq. 4; Dirichlet values stay put."""
    d = disk_nodes(0.06)
    u, f, g = manufactured(d.xy)
    uh, (idx, w, rp, col, val, b) = oracle.poisson_solve(d.xy, d.is_dirichlet, f, g, 2, 12)
    u2 = oracle.explicit_step(idx, w, d.is_dirichlet, f, uh, 1e-6)
    assert np.abs(u2 - uh).max() <= 1e-6 * 1e-6 * np.abs(w).max() * 10
    rng = np.random.default_rng(2)
    u1 = rng.standard_normal(d.N)
    u3 = oracle.explicit_step(idx, w, d.is_dirichlet, f, u1, 1e-6)
    dm = d.is_dirichlet.astype(bool)
    assert np.array_equal(u3[dm], u1[dm])
    lap = (w * u1[idx]).sum(axis=1)
    np.testing.assert_allclose(u3[~dm], u1[~dm] + 1e-6 * (f[~dm] + lap[~dm]), rtol=1e-14, atol=1e-14)


# -------------------------------------------------------------- fixture ------
def test_fixture_counts_and_determinism():
    a, b = disk_nodes(0.04), disk_nodes(0.04)
    assert np.array_equal(a.xy, b.xy)
    assert a.n_boundary == round(2 * math.pi / 0.04)
    assert abs(a.N - math.pi / 0.04 ** 2) < 0.05 * a.N
    r = np.hypot(a.xy[:, 0], a.xy[:, 1])
    assert np.all(r[: a.n_interior] < 1 - 0.02) and np.allclose(r[a.n_interior:], 1.0)
    u = uniform01(splitmix64(1, 1000))
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.05


def test_weights_coincident_nodes_flagged_singular():
    """Two nodes at one point give two identical rows: every stencil that
    holds both is singular (status 1, zero weights); the others are not."""
    d = disk_nodes(0.1)
    xy = d.xy.copy()
    xy[5] = xy[4]
    idx = oracle.knn(xy, 12)
    w, st = oracle.weights(xy, idx, 2)
    holds_both = np.array([(4 in row) and (5 in row) for row in idx])
    assert np.array_equal(st.astype(bool), holds_both)
    assert np.all(w[holds_both] == 0.0)


def test_weights_rank_deficient_stencil_flagged():
    """All nodes on one line: P (monomials to degree 2) has rank 3 < 6, so every
    system is singular; a jittered disk has no such stencil."""
    t = np.linspace(-1.0, 1.0, 40)
    xy = np.ascontiguousarray(np.stack([t, 0.5 * t], axis=1))
    w, st = oracle.weights(xy, oracle.knn(xy, 12), 2)
    assert st.all() and np.all(w == 0.0)
    d = disk_nodes(0.08)
    _, st = oracle.weights(d.xy, oracle.knn(d.xy, 56), 6)
    assert not st.any()


# ------------------------------------------- full-size oracle machinery -----
@pytest.mark.parametrize("h,n,jitter", [(0.02, 56, 0.25), (0.02, 12, 0.25), (1.0 / 32, 30, 0.0), (0.05, 56, 0.0)])
def test_knn_grid_equals_brute_force(h, n, jitter):
    """The cell-grid search returns the brute force's rows exactly (order and
    ties included), on jittered disks and on unjittered grids (exact ties)."""
    d = disk_nodes(h, jitter=jitter)
    assert np.array_equal(oracle.knn_grid(d.xy, n), oracle.knn(d.xy, n))


def test_knn_grid_clustered_and_duplicate_points():
    """Strongly non-uniform density (clusters, exact duplicates, a lone far
    point): the ring bound still decides, or the brute force takes over."""
    rng = np.random.default_rng(7)
    pts = [rng.normal(c, s, size=(k, 2)) for c, s, k in (((0.0, 0.0), 1e-3, 400), ((0.5, 0.2), 0.05, 300),
                                                             ((-0.7, 0.6), 0.2, 200))]
    xy = np.concatenate(pts + [np.array([[5.0, 5.0]]), pts[0][:20]])
    for n in (8, 30):
        assert np.array_equal(oracle.knn_grid(xy, n), oracle.knn(xy, n))


def test_knn_grid_sampled_at_2e5_nodes():
    """At N = 2e5 (a 200k-node disk), 400 seeded queries: grid search = brute force."""
    from fixtures import h_for_nodes

    d = disk_nodes(h_for_nodes(2e5))
    q = (uniform01(splitmix64(11, 400)) * d.N).astype(np.int64)
    assert np.array_equal(oracle.knn_grid(d.xy, 56, q), oracle.knn_query(d.xy, 56, q))


def test_residual_extended_is_the_exact_residual_rounded():
    """b - A x with products and sums in extended precision equals the exact
    rational residual rounded to double, on rows built to cancel badly in
    plain double arithmetic."""
    from fractions import Fraction

    rng = np.random.default_rng(3)
    N, k = 40, 6
    row_ptr = np.arange(0, N * k + 1, k, dtype=np.int64)
    col = rng.integers(0, N, size=N * k).astype(np.int32)
    val = rng.normal(size=N * k) * 1e6
    x = rng.normal(size=N)
    exact_ax = [sum(Fraction(float(val[a])) * Fraction(float(x[col[a]])) for a in range(row_ptr[i], row_ptr[i + 1]))
                for i in range(N)]
    b = np.array([float(v) for v in exact_ax]) + rng.normal(size=N) * 1e-9  # residual ~1e-9 against |Ax| ~1e6
    r = oracle.residual_extended(row_ptr, col, val, x, b)
    exact = np.array([float(Fraction(float(b[i])) - exact_ax[i]) for i in range(N)])
    # long double keeps ~64 bits: the residual to ~2^-64 * sum |a x| ~ 1e-12 absolute here
    assert np.abs(r - exact).max() <= 1e-11 * np.abs(exact).max() + 4e-13
    plain = b - to_scipy(row_ptr, col, val, N) @ x
    assert np.abs(plain - exact).max() > np.abs(r - exact).max()  # double arithmetic loses more


def test_gmres_right_matches_dense_solve():
    """Restarted right-preconditioned GMRES against LAPACK on a small
    nonsymmetric system, with and without a (diagonal) preconditioner."""
    rng = np.random.default_rng(5)
    N = 120
    A = np.eye(N) * 4 + rng.normal(size=(N, N)) * 0.2
    b = rng.normal(size=N)
    ref = np.linalg.solve(A, b)
    for ps in (lambda v: v, lambda v: v / np.diag(A)):
        x, its = oracle.gmres_right(lambda v: A @ v, ps, b, 1e-13, restart=25)
        assert np.abs(x - ref).max() <= 1e-11 * np.abs(ref).max() and its > 0


@pytest.mark.parametrize("h,m,n", [(0.02, 6, 56), (0.012, 4, 30)])
def test_solve_refined_matches_refined_superlu(h, m, n):
    """The Krylov path of solve_refined (GMRES corrections preconditioned by the
    degree-2, 12-node operator) and SuperLU of A itself with the same
    extended-precision refinement reach the same u and lambda to 1e-12; the
    unrefined direct solve agrees to its own forward error (1e-8)."""
    d = disk_nodes(h)
    u_ex, f, g = manufactured(d.xy)
    A = oracle.assemble(oracle.knn_grid(d.xy, n), oracle.weights(d.xy, oracle.knn_grid(d.xy, n), m)[0],
                        d.is_dirichlet)
    idx12 = oracle.knn_grid(d.xy, 12)
    Mp = oracle.assemble(idx12, oracle.weights(d.xy, idx12, 2)[0], d.is_dirichlet)
    b = oracle.rhs(f, g, d.is_dirichlet)
    x_k, info_k = oracle.solve_refined(*A, b, Mp)
    x_d, info_d = oracle.solve_refined(*A, b, None)
    assert np.abs(x_k - x_d).max() <= 1e-12 * np.abs(x_d).max()
    assert info_k["rel_residual"] <= 1e-12 and info_d["rel_residual"] <= 1e-12
    assert np.abs(x_k - oracle.solve_direct(*A, b)).max() <= 1e-8 * np.abs(x_d).max()
    rhs_t = np.where(d.is_dirichlet == 0, np.sin(3 * d.xy[:, 0]), 0.0)
    l_k, _ = oracle.solve_refined(*A, rhs_t, Mp, transpose=True)
    l_d = oracle.solve_direct(*A, rhs_t, transpose=True)
    l_r, _ = oracle.solve_refined(*A, rhs_t, None, transpose=True)
    assert np.abs(l_k - l_r).max() <= 1e-12 * np.abs(l_r).max()
    assert np.abs(l_k - l_d).max() <= 1e-8 * np.abs(l_r).max()


@pytest.mark.parametrize("m,n,bar", [(2, 6, 1e-9), (4, 15, 1e-6)])
def test_weights_unisolvent_against_exact_rational_solution(m, n, bar):
    """n = s: P^T w = lap p alone fixes the weights; solved exactly in rational
    arithmetic from the same shifted coordinates (tests/exact_unisolvent.py).
    The oracle's LU of the whole (n+s)^2 system stays within `bar` of it
    (it loses ~cond(P) ulps: 2.8e-8 with x86 LAPACK, 5.4e-7 with aarch64's,
    at m = 4, n = 15 on this disk)."""
    from exact_unisolvent import exact_weights

    d = disk_nodes(0.1)
    idx = oracle.knn(d.xy, n)
    nodes = np.arange(0, d.N, 3)
    w, st = oracle.weights(d.xy, idx, m, nodes=nodes)
    ex = np.array([exact_weights(d.xy, idx[i], i, m) for i in nodes])
    assert not st.any()
    assert (np.abs(w - ex).max(axis=1) / np.abs(ex).max(axis=1)).max() <= bar
    # and the exact weights are Laplacian-exact on the monomials (Pins the helper too.)
    X = d.xy[idx[nodes[0]]] - d.xy[nodes[0]]
    for a, b in oracle.monomial_exponents(m):
        want = 2.0 if (a, b) in ((2, 0), (0, 2)) else 0.0
        got = float(np.sum(ex[0] * X[:, 0] ** a * X[:, 1] ** b))
        assert abs(got - want) <= 1e-9 * np.abs(ex[0] * X[:, 0] ** a * X[:, 1] ** b).sum() + 1e-12
