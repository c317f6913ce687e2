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


def test_noalloc_at_its_node_limit_against_the_oracle(lib):
    """N = 2^20 nodes, the array's limit (a disk of exactly that many seeded
    nodes), n = 128 and n = 12: sampled rows against the oracle's stencils."""
    import oracle
    from fixtures import sample_indices

    from paper_2107_03632_gb300 import rbffd

    N = 1 << 20
    u = uniform01(splitmix64(2024, 4 * N)).reshape(2 * N, 2)
    pts = 2.0 * u - 1.0
    xy_np = np.ascontiguousarray(pts[(pts * pts).sum(axis=1) < 1.0][:N])
    assert xy_np.shape[0] == N
    xy = torch.from_numpy(xy_np).to(DEV)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    q = sample_indices(N, 2000, 77)
    for n in (128, 12):
        idx = torch.full((N, n), -7, dtype=torch.int32, device=DEV)
        st = lib.rbffd_stencils_noalloc(ctypes.c_void_p(xy.data_ptr()), N, n, ctypes.c_void_p(idx.data_ptr()),
                                        ctypes.c_void_p(stream))
        assert st == 0, rbffd.STATUS_NAMES.get(st, st)
        torch.cuda.synchronize()
        got = idx[torch.from_numpy(q).to(DEV)].cpu().numpy()
        assert np.array_equal(got, oracle.knn_grid(xy_np, n, q))
        assert np.array_equal(got[:16], oracle.knn_query(xy_np, n, q[:16]))
        del idx
    # one node more is refused
    assert lib.rbffd_stencils_noalloc(ctypes.c_void_p(xy.data_ptr()), N + 1, 12, ctypes.c_void_p(0x2000),
                                      ctypes.c_void_p(stream)) == 1


def test_noalloc_inside_a_stream_capture(lib):
    """After one call outside (the address look-up), the entry point is
    captured into a CUDA graph on a side stream and replayed on two node sets
    copied into the same input buffer; each replay equals rbffd_stencils."""
    from paper_2107_03632_gb300 import rbffd

    n = 30
    a = disk_nodes(0.03).xy
    b = np.ascontiguousarray(a[::-1] * 0.9 + 0.01)
    N = a.shape[0]
    xin = torch.from_numpy(a).to(DEV)
    idx = torch.zeros((N, n), dtype=torch.int32, device=DEV)
    side = torch.cuda.Stream(DEV)
    with torch.cuda.stream(side):
        assert lib.rbffd_stencils_noalloc(ctypes.c_void_p(xin.data_ptr()), N, n, ctypes.c_void_p(idx.data_ptr()),
                                          ctypes.c_void_p(side.cuda_stream)) == 0
    side.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        st = lib.rbffd_stencils_noalloc(ctypes.c_void_p(xin.data_ptr()), N, n, ctypes.c_void_p(idx.data_ptr()),
                                        ctypes.c_void_p(side.cuda_stream))
    assert st == 0
    for pts in (a, b):
        xin.copy_(torch.from_numpy(pts))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(idx, rbffd.rbffd_stencils(torch.from_numpy(pts).to(DEV), n))
