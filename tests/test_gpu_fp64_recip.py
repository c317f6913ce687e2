"""The weight solves' FP64 reciprocal and reciprocal square root (float32
seeds moved in and out of doubles by integer instructions, then one
FMA-based correction of third order) against IEEE results computed on the
host: within two ulps (three for the root) for 2^-100 <= |x| < 2^101, and
the IEEE operation itself outside that range."""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_rcp64_rsqrt64_within_two_ulps(lib):
    rng = np.random.default_rng(5)
    mag = np.exp(rng.uniform(np.log(1e-29), np.log(1e29), 200000))
    x = np.concatenate([mag, -mag[:50000], [1.0, 2.0, 0.5, 3.0, 1e-30 * 1.0001, 1e30 * 0.9999]])
    xt = torch.from_numpy(x).to(DEV)
    rcp = torch.empty_like(xt)
    rsq = torch.empty_like(xt)
    assert lib.rbffd_diag_recip(ctypes.c_void_p(xt.data_ptr()), x.size, ctypes.c_void_p(rcp.data_ptr()),
                                ctypes.c_void_p(rsq.data_ptr()), None) == 0
    torch.cuda.synchronize()
    r = rcp.cpu().numpy()
    ref = 1.0 / x
    assert (np.abs(r - ref) <= 2 * np.spacing(np.abs(ref))).all()
    pos = x > 0
    q = rsq.cpu().numpy()[pos]
    # 1/sqrt in float64 carries two roundings: compare within 3 ulps of it
    refq = 1.0 / np.sqrt(x[pos])
    assert (np.abs(q - refq) <= 3 * np.spacing(refq)).all()


def test_outside_float_range_uses_ieee(lib):
    x = np.array([1e-35, 3e-300, 1e35, 7e250, -1e-40, -1e40])
    xt = torch.from_numpy(x).to(DEV)
    rcp = torch.empty_like(xt)
    assert lib.rbffd_diag_recip(ctypes.c_void_p(xt.data_ptr()), x.size, ctypes.c_void_p(rcp.data_ptr()),
                                None, None) == 0
    torch.cuda.synchronize()
    assert np.array_equal(rcp.cpu().numpy(), 1.0 / x)
