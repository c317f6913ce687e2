"""GPU tests of the weight-solve autotuner: whatever configuration it picks
(or is pinned), the weights match the oracle to the parity bar."""

import numpy as np
import pytest
import torch

import oracle
from fixtures import disk_nodes

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("precision", ["fp64", "df", "any"])
@pytest.mark.parametrize("h,m,n,tol", [(0.05, 2, 12, 1e-9), (0.04, 4, 30, 1e-9), (0.06, 6, 56, 1e-7)])
def test_autotuned_and_pinned_configs_match_oracle(lib, h, m, n, tol, precision):
    from paper_2107_03632_gb300 import rbffd

    d = disk_nodes(h)
    xy = torch.from_numpy(d.xy).to(DEV)
    idx_ref = oracle.knn(d.xy, n)
    w_ref, _ = oracle.weights(d.xy, idx_ref, m)
    idx = torch.from_numpy(idx_ref).to(DEV)
    try:
        best = rbffd.rbffd_weights_autotune(xy, idx, m, precision)
        assert best["ms_per_mnode"] > 0 and 1 <= best["warps_per_block"] <= 4
        # the precision selector limits the candidates to FP64 / double-float kernels
        assert {"fp64": "-df" not in best["kernel"], "df": "-df" in best["kernel"], "any": True}[precision]
        got = rbffd.weights_config(n, m)
        assert (got["kernel"], got["warps_per_block"]) == (best["kernel"], best["warps_per_block"])
        w, st = rbffd.rbffd_weights(xy, idx, m)  # the tuned configuration
        err = (np.abs(w.cpu().numpy() - w_ref).max(axis=1) / np.abs(w_ref).max(axis=1)).max()
        assert err <= tol and int(st.sum()) == 0, (best, err)
        if precision != "any":
            return
        for kernel in rbffd.WEIGHTS_KERNELS:  # every pinned configuration
            for wpb in {"null-space-2warp": (2,), "null-space-4warp": (4,), "null-space-df-2warp": (2,),
                        "null-space-df-4warp": (4,)}.get(kernel, (1, 2, 4)):
                try:
                    rbffd.set_weights_config(n, m, kernel, wpb)
                except rbffd.RbffdError:
                    continue  # does not fit in shared memory
                w, st = rbffd.rbffd_weights(xy, idx, m)
                err = (np.abs(w.cpu().numpy() - w_ref).max(axis=1) / np.abs(w_ref).max(axis=1)).max()
                assert err <= tol and int(st.sum()) == 0, (kernel, wpb, err)
    finally:
        rbffd.set_weights_config(n, m, None)
