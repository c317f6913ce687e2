"""Writes the stored oracle references of the full-size parity tests.

Calls only `oracle` and `fixtures` (no GPU, nothing of the CUDA path):

  python tests/golden/make_full_size_reference.py disk_1M_m4_n30 [procs]
  python tests/golden/make_full_size_reference.py disk_4M_m6_n56 [procs]

For the disk workload it builds the oracle's stencils (exact cell-grid search,
identical to the brute force), its weights (one LAPACK solve per stencil,
Sec. II Eq. 1 with the basis of Sec. V), the assembled system (Sec. IV, Eqs.
2-4 at steady state), and solves it with `oracle.solve_refined` (iterative
refinement with an extended-precision residual; corrections by GMRES
preconditioned with the degree-2, 12-node operator of the same nodes), for
the manufactured source u = sin(pi x) sin(pi y).  For the 1M-node disk it
also takes the adjoint gradient of L = sum over interior nodes of
(u - u*)^2, u* the solution for the seeded Fourier source (seed 2108), with
the same machinery on A^T.  A seeded sample of the results goes to
tests/golden/full_size_<workload>.txt (index and value per line, %.17g).
"""

from __future__ import annotations

import math
import multiprocessing as mp
import os
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from fixtures import disk_nodes, fourier_sources, manufactured, sample_indices  # noqa: E402

WORKLOADS = {"disk_1M_m4_n30": (1.7725e-3, 4, 30), "disk_4M_m6_n56": (8.862e-4, 6, 56)}
SEED = 2107
N_SAMPLE = 4096
_G = {}


def _init(path_xy, path_idx):
    _G["xy"] = np.load(path_xy, mmap_mode="r")
    _G["idx"] = np.load(path_idx, mmap_mode="r") if path_idx else None


def _knn_chunk(a):
    n, q = a
    return oracle.knn_grid(np.asarray(_G["xy"]), n, q)


def _weights_chunk(a):
    m, nodes = a
    w, st = oracle.weights(np.asarray(_G["xy"]), _G["idx"], m, nodes=nodes)
    return w, st


def stencils(tmp, xy, n, procs):
    pxy = os.path.join(tmp, "xy.npy")
    np.save(pxy, xy)
    chunks = np.array_split(np.arange(xy.shape[0]), procs * 8)
    with mp.get_context("spawn").Pool(procs, _init, (pxy, None)) as pool:
        return np.concatenate(pool.map(_knn_chunk, [(n, c) for c in chunks]))


def weights(tmp, xy, idx, m, procs):
    pxy, pidx = os.path.join(tmp, "xy.npy"), os.path.join(tmp, "idx.npy")
    np.save(pxy, xy)
    np.save(pidx, idx)
    chunks = np.array_split(np.arange(xy.shape[0]), procs * 32)
    with mp.get_context("spawn").Pool(procs, _init, (pxy, pidx)) as pool:
        res = pool.map(_weights_chunk, [(m, c) for c in chunks])
    w = np.concatenate([r[0] for r in res])
    st = np.concatenate([r[1] for r in res])
    if st.any():
        raise RuntimeError(f"{int(st.sum())} singular stencils")
    return w


def write(path, header, sections):
    with open(path, "w") as fo:
        for ln in header:
            fo.write(f"# {ln}\n")
        for title, ii, vv in sections:
            fo.write(f"[{title}] {ii.size}\n")
            for i, v in zip(ii, vv):
                fo.write(f"{int(i)} {float(v):.17g}\n")


def main():
    name = sys.argv[1]
    procs = int(sys.argv[2]) if len(sys.argv) > 2 else (os.cpu_count() or 1)
    h, m, n = WORKLOADS[name]
    d = disk_nodes(h, SEED)
    u_ex, f, g = manufactured(d.xy)
    log = []
    t0 = time.time()
    with tempfile.TemporaryDirectory() as tmp:
        idx = stencils(tmp, d.xy, n, procs)
        idx12 = stencils(tmp, d.xy, 12, procs)
        log.append(f"stencils {time.time() - t0:.0f} s")
        w = weights(tmp, d.xy, idx, m, procs)
        w12 = weights(tmp, d.xy, idx12, 2, procs)
        log.append(f"weights {time.time() - t0:.0f} s")
    A = oracle.assemble(idx, w, d.is_dirichlet)
    Mp = oracle.assemble(idx12, w12, d.is_dirichlet)
    del idx, w, idx12, w12
    log.append(f"assembly {time.time() - t0:.0f} s")
    b = oracle.rhs(f, g, d.is_dirichlet)
    u, info = oracle.solve_refined(*A, b, Mp)
    log.append(f"solve {time.time() - t0:.0f} s: {info}")
    print(log[-1], flush=True)
    samp = sample_indices(d.N, N_SAMPLE, SEED + 17)
    sections = [("u", samp, u[samp])]
    header = [f"oracle reference for the full-size parity tests: {name}, N = {d.N}, h = {h}, m = {m}, n = {n}, "
              f"seed {SEED}",
              "written by tests/golden/make_full_size_reference.py (oracle and fixtures only)",
              "u: A u = b for the manufactured source (f = 2 pi^2 sin(pi x) sin(pi y), g = u on r = 1),",
              "   by oracle.solve_refined (extended-precision residual refinement, GMRES corrections)",
              f"max |u - sin(pi x) sin(pi y)| = {np.abs(u - u_ex).max():.6e}",
              f"refined relative residual = {info['rel_residual']:.3e}"]
    if name == "disk_1M_m4_n30":
        fstar = fourier_sources(d.xy, 1, SEED + 1)[0]
        ustar, info_s = oracle.solve_refined(*A, oracle.rhs(fstar, g, d.is_dirichlet), Mp)
        interior = d.is_dirichlet == 0
        dLdu = np.where(interior, 2.0 * (u - ustar), 0.0)
        lam, info_a = oracle.solve_refined(*A, dLdu, Mp, transpose=True)
        loss = float(np.sum((u - ustar)[interior] ** 2))
        log.append(f"adjoint {time.time() - t0:.0f} s: {info_a}")
        print(log[-1], flush=True)
        si = samp[interior[samp]]
        bnd = np.nonzero(~interior)[0]
        sb = bnd[sample_indices(bnd.size, 1024, SEED + 18)]
        sections += [("ustar", samp, ustar[samp]), ("dLdf", si, -lam[si]), ("dLdg", sb, lam[sb])]
        header += ["ustar: the same with f* = the seeded Fourier source (fixtures.fourier_sources, seed 2108)",
                   f"L = sum over interior nodes of (u - ustar)^2 = {loss:.17g}",
                   "dLdf = -lambda (interior nodes), dLdg = lambda (Dirichlet nodes), A^T lambda = 2 (u - ustar)",
                   f"refined relative residuals: ustar {info_s['rel_residual']:.3e}, "
                   f"lambda {info_a['rel_residual']:.3e}"]
    header += ["timings: " + "; ".join(x.split(":")[0] for x in log)]
    write(os.path.join(os.path.dirname(os.path.abspath(__file__)), f"full_size_{name}.txt"), header, sections)


if __name__ == "__main__":
    main()
