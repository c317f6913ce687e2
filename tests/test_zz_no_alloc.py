"""rbffd_stencils_noalloc: stencils for callers that cannot allocate.

Some callers cannot call cudaMalloc (or anything that allocates) on their
path -- code inside a CUDA stream capture, an arena that owns all device
memory, a loop that must not allocate -- and cannot pass a workspace
either.  The no-alloc entry point keeps its scratch in a fixed device array
inside the library.  Its results must equal those of rbffd_stencils (with
a caller workspace) bit for bit, on consecutive calls that reuse the same
array, and sizes beyond the array's limit must be refused up front.

This file is collected last so that a failure here does not hide others.
"""

import ctypes

import numpy as np
import pytest
import torch

from fixtures import disk_nodes, splitmix64, uniform01

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _cases():
    d = disk_nodes(0.02)
    u = uniform01(splitmix64(91, 2 * 5000)).reshape(5000, 2)
    return [(d.xy, 30), (np.ascontiguousarray(2.0 * u - 1.0), 12), (d.xy, 56)]


def test_noalloc_matches_workspace_version_on_consecutive_calls(lib):
    from paper_2107_03632_gb300 import rbffd

    stream = torch.cuda.current_stream(DEV).cuda_stream
    for xy_np, n in _cases():
        xy = torch.from_numpy(xy_np).to(DEV)
        N = xy.shape[0]
        idx = torch.full((N, n), -7, dtype=torch.int32, device=DEV)
        st = lib.rbffd_stencils_noalloc(ctypes.c_void_p(xy.data_ptr()), N, n, ctypes.c_void_p(idx.data_ptr()),
                                        ctypes.c_void_p(stream))
        assert st == 0, rbffd.STATUS_NAMES.get(st, st)
        ref = rbffd.rbffd_stencils(xy, n)
        torch.cuda.synchronize()
        assert torch.equal(idx, ref)


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    limit = 1 << 20
    # refused before anything touches the device (the pointers are never read)
    assert lib.rbffd_stencils_noalloc(ctypes.c_void_p(0x1000), limit + 1, 12, ctypes.c_void_p(0x2000), None) == 1
    assert lib.rbffd_stencils_noalloc(ctypes.c_void_p(0x1000), 0, 12, ctypes.c_void_p(0x2000), None) == 1
