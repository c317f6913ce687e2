"""Every stage of the CUDA path through the bounds-checked library, on small
node sets, against the oracle.

Run as its own process with RBFFD_CHECKED=1 (the package then loads
librbffd_checked.so, in which every computed index is tested before its
access and a violation is recorded instead of performed).  After each stage
the device is synchronised and the violation records are read and cleared.
Prints one JSON object: per stage the violations (and the first one's site)
and the parity figures; "failures" lists what broke a bar.  The bars are the
ones of the normal build's parity tests: stencils and assembly bit-exact,
weights 1e-9 (m <= 4) and 1e-7 (m = 6) relative per stencil, 1e-6 for the
double-float kernels, solutions 1e-8 relative to the oracle's direct solve.
"""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from fixtures import disk_nodes, fourier_sources, manufactured  # noqa: E402
from oracle.assemble import to_scipy  # noqa: E402
from paper_2107_03632_gb300 import rbffd  # noqa: E402

DEV = "cuda:0"
REPORT = {"stages": {}, "failures": []}


def T(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def rel_rowwise(w, w_ref):
    num = np.abs(w - w_ref).max(axis=1)
    den = np.abs(w_ref).max(axis=1)
    return float((num / den).max())


def rel(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


def stage(name, expect_violations=0, **figures):
    """Reads and clears the violation records after the stage's work."""
    torch.cuda.synchronize()
    r = rbffd.rbffd_checked_read(reset=True)
    entry = dict(figures)
    entry["violations"] = r["violations"]
    if r["violations"]:
        entry["first"] = {k: r[k] for k in ("file", "line", "index", "bound")}
    REPORT["stages"][name] = entry
    if r["violations"] != expect_violations:
        REPORT["failures"].append(f"{name}: {r['violations']} violations, expected {expect_violations}")
    return r


def bar(name, value, limit):
    if not (value <= limit):
        REPORT["failures"].append(f"{name}: {value} > {limit}")


def probes():
    """The checker itself: an in-range access, then one out-of-range access
    of each kind, each recorded and redirected."""
    v = rbffd.rbffd_checked_probe(3, 8, 2, 6, 56).item()
    stage("probe in range", value=v)
    bar("probe in range value", abs(v - 1.0), 0.0)
    cases = [("probe index", (9, 8, 0, 0, 0), (9, 8)), ("probe negative index", (-1, 8, 0, 0, 0), (-1, 8)),
             ("probe span", (0, 8, 5, 4, 0), (9, 8)), ("probe shared memory", (0, 8, 0, 0, 64), (64, 64))]
    for name, args, (index, bound) in cases:
        rbffd.rbffd_checked_probe(*args)
        r = stage(name, expect_violations=(2 if name == "probe shared memory" else 1))
        if r["file"] != "api.cu" or r["index"] != index or r["bound"] != bound:
            REPORT["failures"].append(f"{name}: recorded {r}")


def stencils_and_weights():
    for h, n in ((0.25, 12), (0.1, 30), (0.08, 56), (0.04, 100)):
        d = disk_nodes(h, seed=3)
        idx = rbffd.rbffd_stencils(T(d.xy), n).cpu().numpy()
        ok = bool(np.array_equal(idx, oracle.knn(d.xy, n)))
        stage(f"stencils N={d.N} n={n}", bitexact=ok)
        if not ok:
            REPORT["failures"].append(f"stencils N={d.N} n={n} differ")
    # the noalloc entry (its scratch is a file-scope device array)
    d = disk_nodes(0.1, seed=4)
    idx = torch.empty((d.N, 12), dtype=torch.int32, device=DEV)
    xy = T(d.xy)
    st = rbffd.load().rbffd_stencils_noalloc(rbffd._ptr(xy), d.N, 12, rbffd._ptr(idx), rbffd._stream(idx.device))
    ok = st == 0 and bool(np.array_equal(idx.cpu().numpy(), oracle.knn(d.xy, 12)))
    stage("stencils noalloc", bitexact=ok)
    if not ok:
        REPORT["failures"].append("stencils noalloc differ")
    # every weight kernel, every degree it takes
    cases = [(0.1, 0, 5), (0.1, 2, 12), (0.08, 4, 30), (0.08, 6, 56), (0.15, 8, 90)]
    for h, m, n in cases:
        d = disk_nodes(h, seed=5)
        idx = oracle.knn(d.xy, n)
        w_ref, _ = oracle.weights(d.xy, idx, m)
        for kernel in rbffd.WEIGHTS_KERNELS:
            df = "df" in kernel
            if (m == 0 and kernel != "gauss") or (df and not 1 <= m <= 6):
                continue
            if ("half" in kernel or "quarter" in kernel) and (m > 4 or n > 32):
                continue
            # warps per block: 1 for the one-warp kernels, 2 / 4 for the
            # two- and four-warp ones, 2 for the half- and quarter-warp ones
            wpb = 4 if "4warp" in kernel else (2 if ("2warp" in kernel or "half" in kernel or "quarter" in kernel)
                                               else 1)
            try:
                rbffd.set_weights_config(n, m, kernel, wpb)
            except rbffd.RbffdError as e:  # does not fit in shared memory at this (n, m)
                REPORT["stages"][f"weights {kernel} m={m} n={n}"] = {"skipped": str(e)}
                continue
            w, status = rbffd.rbffd_weights(T(d.xy), T(idx), m)
            err = rel_rowwise(w.cpu().numpy(), w_ref)
            stage(f"weights {kernel} m={m} n={n}", err=err)
            bar(f"weights {kernel} m={m} n={n}", err, 1e-6 if df else (1e-7 if m >= 6 else 1e-9))
            rbffd.set_weights_config(n, m, None)
    d = disk_nodes(0.08, seed=6)
    idx = T(oracle.knn(d.xy, 30))
    best = rbffd.rbffd_weights_autotune(T(d.xy), idx, 4, precision="any")
    stage("weights autotune", best=best["kernel"])
    rbffd.set_weights_config(30, 4, None)


def system(h, m, n, seed):
    d = disk_nodes(h, seed=seed)
    u, f, g = manufactured(d.xy)
    idx = rbffd.rbffd_stencils(T(d.xy), n)
    w, _ = rbffd.rbffd_weights(T(d.xy), idx, m)
    mask = T(d.is_dirichlet)
    A = rbffd.rbffd_assemble(idx, w, mask, want_f32=True)
    b = rbffd.rbffd_rhs(T(f), T(g), mask)
    return d, f, g, idx, w, mask, A, b


def assembly_and_solves():
    for h, m, n in ((0.05, 2, 12), (0.04, 4, 30), (0.06, 6, 56)):
        d, f, g, idx, w, mask, A, b = system(h, m, n, 7)
        rp, col, val = oracle.assemble(idx.cpu().numpy(), w.cpu().numpy(), d.is_dirichlet)
        ok = (np.array_equal(A.row_ptr.cpu().numpy(), rp) and np.array_equal(A.col.cpu().numpy(), col)
              and np.array_equal(A.val.cpu().numpy(), val))
        b_ref = oracle.rhs(f, g, d.is_dirichlet)
        ok = ok and np.array_equal(b.cpu().numpy(), b_ref)
        stage(f"assembly m={m} n={n}", bitexact=bool(ok))
        if not ok:
            REPORT["failures"].append(f"assembly m={m} n={n} differs")
        AT = rbffd.rbffd_transpose(A, want_f32=True)
        S = to_scipy(rp, col, val, d.N).T.tocsr()
        S.sort_indices()
        ok = (np.array_equal(AT.row_ptr.cpu().numpy(), S.indptr) and np.array_equal(AT.col.cpu().numpy(), S.indices)
              and np.array_equal(AT.val.cpu().numpy(), S.data))
        stage(f"transpose m={m} n={n}", bitexact=bool(ok))
        if not ok:
            REPORT["failures"].append(f"transpose m={m} n={n} differs")
        ref = oracle.solve_direct(rp, col, val, b_ref)
        for precision in ("fp64", "mixed"):
            x, info = rbffd.rbffd_solve(A, b, opts=rbffd.make_opts(tol=1e-10, precision=precision))
            err = rel(x.cpu().numpy(), ref)
            stage(f"solve jacobi {precision} m={m} n={n}", err=err, iters=info["iters"])
            bar(f"solve jacobi {precision} m={m} n={n}", err, 1e-8)
        fwd = rbffd.Multigrid(T(d.xy), mask, A)
        stage(f"multigrid setup m={m} n={n}", levels=fwd.levels())
        for precision in ("fp64", "mixed"):
            x, info = rbffd.rbffd_solve(A, b, opts=rbffd.make_opts(tol=1e-10, precision=precision, mg=fwd))
            err = rel(x.cpu().numpy(), ref)
            stage(f"solve multigrid {precision} m={m} n={n}", err=err, iters=info["iters"])
            bar(f"solve multigrid {precision} m={m} n={n}", err, 1e-8)
        # adjoint: misfit gradient, then A^T lambda = dL/du with each adjoint hierarchy
        ut = T(ref * 0.5)
        dLdu = rbffd.rbffd_misfit_grad(T(ref), ut, mask)
        _, _, lam_ref = oracle.adjoint_gradient(rp, col, val, d.is_dirichlet, dLdu.cpu().numpy())
        hiers = {"transposed": rbffd.Multigrid.adjoint_of(fwd, AT),
                 "galerkin": rbffd.Multigrid.galerkin_adjoint_of(fwd, AT)}
        stage(f"adjoint hierarchies m={m} n={n}")
        for name, hier in hiers.items():
            lam, _, _, info = rbffd.rbffd_solve_adjoint(AT, mask, dLdu,
                                                        opts=rbffd.make_opts(tol=1e-11, precision="mixed", mg=hier))
            err = rel(lam.cpu().numpy(), lam_ref)
            stage(f"adjoint {name} m={m} n={n}", err=err, iters=info["iters"])
            bar(f"adjoint {name} m={m} n={n}", err, 1e-8)
        # explicit time loop
        fe = np.ascontiguousarray(f)
        u0 = np.where(d.is_dirichlet, g, 0.0)
        loop = rbffd.ExplicitLoop(idx, w, mask)
        dt = 1e-6
        uref = u0.copy()
        for _ in range(5):
            uref = oracle.explicit_step(idx.cpu().numpy(), w.cpu().numpy(), d.is_dirichlet, fe, uref, dt)
        ug = loop.run(T(fe), T(u0), dt, 5)
        err = rel(ug.cpu().numpy(), uref)
        stage(f"explicit m={m} n={n}", err=err)
        bar(f"explicit m={m} n={n}", err, 1e-12)


def batched(n_rhs):
    """n_rhs odd: one right-hand side per lane and half-warp; even: two
    adjacent ones per lane (8- and 16-byte accesses)."""
    specs = [(0.1, 2, 12), (0.12, 6, 56), (0.08, 4, 30)]
    nodes, masks, fs, gs, sizes = [], [], [], [], []
    for k, (h, m, n) in enumerate(specs):
        d = disk_nodes(h, seed=40 + k)
        F = fourier_sources(d.xy, n_rhs, 140 + k).T
        _, fman, gman = manufactured(d.xy)
        F[:, 0] = fman
        G = np.zeros_like(F)
        G[:, 0] = gman
        nodes.append(d.xy)
        masks.append(d.is_dirichlet)
        fs.append(F)
        gs.append(G)
        sizes.append((d.N, m, n))
    xy, mask, F, G = (np.concatenate(a) for a in (nodes, masks, fs, gs))
    refs = []
    off = 0
    for N, m, n in sizes:
        sl = slice(off, off + N)
        idx = oracle.knn(xy[sl], n)
        w, _ = oracle.weights(xy[sl], idx, m)
        rp, col, val = oracle.assemble(idx, w, mask[sl])
        refs.append([oracle.solve_direct(rp, col, val, oracle.rhs(F[sl, k], G[sl, k], mask[sl]))
                     for k in range(n_rhs)])
        off += N
    modes = {"jacobi": (0, 0, 0), "mg": (1, 0, 0), "mg-persistent": (1, 1, 0), "mg-device-loop": (1, 0, 1)}
    for mode, (precond, persistent, device_loop) in modes.items():
        opts = rbffd.make_opts(precision="mixed", tol=1e-10)
        opts.precond, opts.persistent, opts.device_loop = precond, persistent, device_loop
        u, infos, st = rbffd.rbffd_solve_batched(sizes, T(xy), T(mask), T(F), T(G), opts=opts)
        u = u.cpu().numpy()
        err = 0.0
        off = 0
        for (N, m, n), ref in zip(sizes, refs):
            for k in range(n_rhs):
                err = max(err, rel(u[off:off + N, k], ref[k]))
            off += N
        stage(f"batched {mode} rhs={n_rhs}", err=err, status=int(st))
        bar(f"batched {mode} rhs={n_rhs}", err, 1e-8)
        if st != 0:
            REPORT["failures"].append(f"batched {mode} rhs={n_rhs}: status {st}")


def main():
    lib = rbffd.load()
    assert rbffd.lib_path().endswith("librbffd_checked.so"), rbffd.lib_path()
    first = rbffd.rbffd_checked_read(reset=True)
    REPORT["checked"] = first["checked"]
    if first["checked"] != 1:
        REPORT["failures"].append("the loaded library is not the checked build")
    del lib
    parts = (probes, stencils_and_weights, assembly_and_solves, lambda: batched(3), lambda: batched(4))
    for part in parts:
        try:
            part()
        except Exception as e:  # report, do not hide
            REPORT["failures"].append(f"{getattr(part, '__name__', 'part')}: {type(e).__name__}: {e}")
    print(json.dumps(REPORT))
    return 0


if __name__ == "__main__":
    sys.exit(main())
