"""Parity at the workloads' full sizes, in the benchmark's launch configuration.

1M nodes (m = 4, n = 30) and 4M nodes (m = 6, n = 56), seeded disks:

* stencils: 10^4 seeded sampled rows bit-exact against the oracle's grid
  search (itself pinned to the brute force) and 64 against the brute force;
* weights: the same rows against the oracle's per-stencil LAPACK solves, for
  the FP64 default and for the double-float kernels, at 1e-9 (m <= 4) and
  1e-7 (m = 6) relative max-norm per stencil;
* solution: u from the benchmark's step (multigrid-preconditioned BiCGSTAB to
  relative residual 1e-10, float32 and FP64 V-cycles) against the oracle's
  own solution of its own system (tests/golden/full_size_*.txt, written by
  tests/golden/make_full_size_reference.py with oracle.solve_refined) at
  4096 sampled nodes, 1e-8 relative max-norm;
* at 1M nodes, the differentiable solve: the GPU adjoint
  gradient of L = sum over interior nodes of (u - u*)^2 against the oracle's
  adjoint gradient at sampled nodes, and against central differences of L
  along 32 seeded directions of (f, g).
"""

import os

import numpy as np
import pytest
import torch

import oracle
from conftest import ROOT
from fixtures import disk_nodes, fourier_sources, manufactured, sample_indices

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SEED = 2107
CASES = {"disk_1M_m4_n30": (1.7725e-3, 4, 30, 1e-9), "disk_4M_m6_n56": (8.862e-4, 6, 56, 1e-7)}


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def golden(name):
    """Sections of tests/golden/full_size_<name>.txt: {title: (indices, values)}."""
    out, cur = {}, None
    for line in open(os.path.join(ROOT, "tests", "golden", f"full_size_{name}.txt")):
        if line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line[1 : line.index("]")]
            out[cur] = ([], [])
            continue
        i, v = line.split()
        out[cur][0].append(int(i))
        out[cur][1].append(float(v))
    return {k: (np.array(a, dtype=np.int64), np.array(b)) for k, (a, b) in out.items()}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, lib):
    from paper_2107_03632_gb300 import rbffd

    name = request.param
    h, m, n, wtol = CASES[name]
    d = disk_nodes(h, SEED)
    u_ex, f, g = manufactured(d.xy)
    xy, mask = T(d.xy), T(d.is_dirichlet)
    idx = rbffd.rbffd_stencils(xy, n)
    rbffd.set_weights_config(n, m, None)  # the library default: FP64
    w, st = rbffd.rbffd_weights(xy, idx, m)
    q = sample_indices(d.N, 10000, SEED + 31)
    yield dict(name=name, h=h, m=m, n=n, wtol=wtol, d=d, f=f, g=g, u_ex=u_ex, xy=xy, mask=mask, idx=idx, w=w,
               st=st, q=q, idx_q=idx[T(q)].cpu().numpy())
    torch.cuda.empty_cache()


def test_full_size_stencils_sampled(case):
    d, n, q = case["d"], case["n"], case["q"]
    assert q.size == 10000
    ref = oracle.knn_grid(d.xy, n, q)
    assert np.array_equal(case["idx_q"], ref)
    qb = q[:64]
    assert np.array_equal(case["idx_q"][:64], oracle.knn_query(d.xy, n, qb))


def _rel_rows(w, ref):
    return (np.abs(w - ref).max(axis=1) / np.abs(ref).max(axis=1)).max()


def test_full_size_weights_sampled(case):
    """FP64 (the default the benchmark times) and the double-float kernels."""
    from paper_2107_03632_gb300 import rbffd

    d, m, n, q = case["d"], case["m"], case["n"], case["q"]
    ref, st_ref = oracle.weights_rows(d.xy, oracle.knn_grid(d.xy, n, q), q, m)
    assert int(st_ref.sum()) == 0 and int(case["st"].sum().item()) == 0
    assert rbffd.weights_config(n, m)["kernel"].find("-df") < 0
    err64 = _rel_rows(case["w"][T(q)].cpu().numpy(), ref)
    print(f"{case['name']}: sampled weights, FP64 default: {err64:.3e}")
    assert err64 <= case["wtol"], err64
    try:
        for kernel, wpb in (("null-space-df", 1), ("null-space-df-4warp", 4)):
            rbffd.set_weights_config(n, m, kernel, wpb)
            w, st = rbffd.rbffd_weights(case["xy"], case["idx"], m)
            errdf = _rel_rows(w[T(q)].cpu().numpy(), ref)
            print(f"{case['name']}: sampled weights, {kernel}: {errdf:.3e}")
            assert errdf <= case["wtol"] and int(st.sum().item()) == 0, (kernel, errdf)
            del w, st
    finally:
        rbffd.set_weights_config(n, m, None)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_solution_vs_oracle(case, precision):
    """u of the benchmark's solve (FP64 weights) at tol 1e-10 against the
    oracle's solution of its own system, at the stored sampled nodes."""
    from paper_2107_03632_gb300 import rbffd

    ref_i, ref_u = golden(case["name"])["u"]
    A = rbffd.rbffd_assemble(case["idx"], case["w"], case["mask"], want_f32=True)
    b = rbffd.rbffd_rhs(T(case["f"]), T(case["g"]), case["mask"])
    mg = rbffd.Multigrid(case["xy"], case["mask"], A)
    x, info = rbffd.rbffd_solve(A, b, opts=rbffd.make_opts(tol=1e-10, precision=precision, inner_tol=1e-10, mg=mg))
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10, info
    u = x.cpu().numpy()
    err = np.abs(u[ref_i] - ref_u).max() / np.abs(ref_u).max()
    print(f"{case['name']}: solution ({precision}), {info['iters']} iterations, relative residual "
          f"{info['rel_residual']:.2e}: {err:.3e} against the oracle")
    assert err <= 1e-8, err
    assert np.abs(u - case["u_ex"]).max() <= 1e-5  # the discretisation error of the scheme
    del A, b, mg, x


@pytest.mark.parametrize("hierarchy", ["transposed", "galerkin"])
def test_full_size_adjoint_gradient(case, hierarchy):
    """The differentiable solve at 1M nodes: forward solve, misfit gradient,
    adjoint solve (with either adjoint hierarchy) -- against the oracle's
    adjoint gradient at the stored sampled nodes, and (once) against central
    differences of L."""
    from paper_2107_03632_gb300 import rbffd

    if case["name"] != "disk_1M_m4_n30":
        pytest.skip("the differentiable solve is the 1M-node workload")
    gold = golden(case["name"])
    d, m, n = case["d"], case["m"], case["n"]
    A = rbffd.rbffd_assemble(case["idx"], case["w"], case["mask"], want_f32=True)
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    mg = rbffd.Multigrid(case["xy"], case["mask"], A)
    mga = (rbffd.Multigrid.galerkin_adjoint_of if hierarchy == "galerkin" else rbffd.Multigrid.adjoint_of)(mg, AT)
    opts = rbffd.make_opts(tol=1e-10, precision="mixed", mg=mg)
    fstar = fourier_sources(d.xy, 1, SEED + 1)[0]
    u, info = rbffd.rbffd_solve(A, rbffd.rbffd_rhs(T(case["f"]), T(case["g"]), case["mask"]), opts=opts)
    ustar, info_s = rbffd.rbffd_solve(A, rbffd.rbffd_rhs(T(fstar), T(case["g"]), case["mask"]), opts=opts)
    dLdu = rbffd.rbffd_misfit_grad(u, ustar, case["mask"])
    lam, dLdf, dLdg, info_a = rbffd.rbffd_solve_adjoint(AT, case["mask"], dLdu,
                                                        opts=rbffd.make_opts(tol=1e-10, precision="mixed", mg=mga))
    assert info["status"] == 0 and info_s["status"] == 0 and info_a["status"] == 0, (info, info_s, info_a)
    # against the oracle's adjoint gradient (its own solves of its own system)
    gf, gg = dLdf.cpu().numpy(), dLdg.cpu().numpy()
    scale = max(np.abs(gold["dLdf"][1]).max(), np.abs(gold["dLdg"][1]).max())
    ef = np.abs(gf[gold["dLdf"][0]] - gold["dLdf"][1]).max() / scale
    eg = np.abs(gg[gold["dLdg"][0]] - gold["dLdg"][1]).max() / scale
    print(f"{case['name']}: adjoint ({hierarchy} hierarchy, {info_a['iters']} iterations): dL/df {ef:.3e}, "
          f"dL/dg {eg:.3e} against the oracle")
    assert max(ef, eg) <= 1e-7, (ef, eg)
    if hierarchy == "galerkin":
        assert info_a["iters"] <= 20, info_a
    assert np.abs(ustar.cpu().numpy()[gold["ustar"][0]] - gold["ustar"][1]).max() <= 1e-8 * np.abs(gold["ustar"][1]).max()
    if hierarchy != "galerkin":
        return  # the central differences below check the gradient once
    # central differences of L along 32 seeded directions v = (v_f, v_g), |v|_inf = 1, eps = 1e-6 |theta|_inf.
    # L is quadratic in theta = (f, g): L(theta +- eps v) uses u(theta +- eps v) = u -+ ... = u +- z with
    # z = A^-1 (b(theta + eps v) - b(theta)) = eps A^-1 b(v_f, v_g), each z a GPU solve of its own right-hand
    # side to relative residual 1e-10, and L(+) - L(-) = sum_interior (u+ - u-)(u+ + u- - 2 u*), the
    # difference of the two squares written out (the two L values agree to ~1e-8 of their size).
    interior = d.is_dirichlet == 0
    uu, us = u.cpu().numpy(), ustar.cpu().numpy()
    theta_inf = max(np.abs(case["f"]).max(), np.abs(case["g"]).max())
    eps = 1e-6 * theta_inf
    rng = np.random.default_rng(2107)
    worst = 0.0
    for _ in range(32):
        v = rng.standard_normal(d.N)
        v /= np.abs(v).max()
        vf, vg = np.where(interior, v, 0.0), np.where(interior, 0.0, v)
        z, info_z = rbffd.rbffd_solve(A, rbffd.rbffd_rhs(T(eps * vf), T(eps * vg), case["mask"]), opts=opts)
        assert info_z["status"] == 0, info_z
        zz = z.cpu().numpy()
        up, um = uu + zz, uu - zz
        fd = np.sum(((up - um) * (up + um - 2.0 * us))[interior]) / (2.0 * eps)
        ad = float(np.dot(gf, vf) + np.dot(gg, vg))
        worst = max(worst, abs(fd - ad) / max(abs(fd), abs(ad)))
    print(f"{case['name']}: central differences, 32 directions: worst relative difference {worst:.3e}")
    assert worst <= 1e-5, worst
    del A, AT, mg, mga
