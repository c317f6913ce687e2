"""The C-ABI library builds, loads and exports every symbol the header declares.

Host-only entry points (status strings, version, workspace sizes) and the
synchronous argument checks are exercised here without a GPU: argument
errors return before anything touches CUDA.
"""

import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "rbffd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(rbffd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def cdll():
    from paper_2107_03632_gb300 import _build, rbffd

    _build.build()
    return rbffd.load()


def test_header_declares_the_pipeline():
    names = declared_functions()
    for must in ["rbffd_stencils", "rbffd_weights", "rbffd_assemble", "rbffd_solve", "rbffd_solve_adjoint",
                 "rbffd_rhs", "rbffd_assemble_pattern", "rbffd_transpose"]:
        assert must in names


def test_every_declared_symbol_is_exported(cdll):
    from paper_2107_03632_gb300 import rbffd

    names = declared_functions()
    assert names, "no declarations parsed"
    for nm in names:
        assert hasattr(cdll, nm), f"{nm} declared in rbffd.h but not exported"
        assert nm in rbffd.SIGNATURES, f"{nm} has no ctypes signature in the binding"
    out = subprocess.run(["nm", "-D", "--defined-only", rbffd.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(rbffd_\w+)\b", out))
    assert set(names) <= exported


def test_no_cuda_driver_dependency_at_load():
    from paper_2107_03632_gb300 import rbffd

    out = subprocess.run(["ldd", rbffd.lib_path()], capture_output=True, text=True).stdout
    assert "libcuda.so" not in out  # the runtime is static; the driver is opened lazily


def test_host_entry_points(cdll):
    assert cdll.rbffd_version() == 100
    assert cdll.rbffd_status_string(0) == b"RBFFD_OK"
    assert cdll.rbffd_status_string(4) == b"RBFFD_ERR_NOT_CONVERGED"
    assert cdll.rbffd_status_string(99) == b"RBFFD_UNKNOWN_STATUS"
    assert cdll.rbffd_stencils_workspace_size(0, 12) == 0
    a = cdll.rbffd_stencils_workspace_size(2000, 12)
    b = cdll.rbffd_stencils_workspace_size(4_000_000, 56)
    assert 0 < a < b
    assert b >= 4_000_000 * (16 + 4 + 4)
    assert cdll.rbffd_assemble_workspace_size(1000) > 0
    assert cdll.rbffd_transpose_workspace_size(1000) >= 4000


def test_solve_workspace_grows_for_mixed(cdll):
    from paper_2107_03632_gb300 import rbffd

    o64 = rbffd.make_opts(precision="fp64")
    o32 = rbffd.make_opts(precision="mixed")
    n = 100_000
    s64 = cdll.rbffd_solve_workspace_size(n, ctypes.byref(o64))
    s32 = cdll.rbffd_solve_workspace_size(n, ctypes.byref(o32))
    assert s64 >= 8 * 8 * n and s32 >= s64 + 2 * 8 * n


def test_argument_errors_return_before_cuda(cdll):
    INVALID, WS = 1, 7
    # null pointers / bad sizes
    assert cdll.rbffd_stencils(None, 10, 4, None, None, 0, None) == INVALID
    assert cdll.rbffd_stencils(0x1000, 10, 11, 0x2000, 0x3000, 1 << 20, None) == INVALID  # n > N
    assert cdll.rbffd_stencils(0x1000, 10, 200, 0x2000, 0x3000, 1 << 20, None) == INVALID  # n > max
    assert cdll.rbffd_stencils(0x1008, 10, 4, 0x2000, 0x3000, 1 << 20, None) == INVALID  # xy not 16-B aligned
    assert cdll.rbffd_stencils(0x1000, 10, 4, 0x2000, 0x3001, 1 << 20, None) == WS  # misaligned workspace
    assert cdll.rbffd_stencils(0x1000, 10, 4, 0x2000, 0x3000, 16, None) == WS  # too small
    # weights: n < s (m = 4 needs 15 nodes), m out of range
    assert cdll.rbffd_weights(0x1000, 0x2000, 100, 12, 4, 0x3000, None, None) == INVALID
    assert cdll.rbffd_weights(0x1000, 0x2000, 100, 12, 9, 0x3000, None, None) == INVALID
    assert cdll.rbffd_weights(None, 0x2000, 100, 12, 2, 0x3000, None, None) == INVALID
    # assembly / rhs
    assert cdll.rbffd_assemble_pattern(None, 10, 4, 0x1000, 0x2000, 1 << 20, None) == INVALID
    assert cdll.rbffd_assemble(None, 0x1, 0x1, 10, 4, 0x1, 10, 0x1, 0x1, None, None) == INVALID
    assert cdll.rbffd_rhs(None, 0x1, 0x1, 10, 0x1, None) == INVALID


def test_solve_argument_errors(cdll):
    from paper_2107_03632_gb300 import rbffd

    A = rbffd.Csr(10, 30, 0x1000, 0x2000, 0x3000, 0)
    info = rbffd.SolveInfo()
    bad_tol = rbffd.make_opts(tol=0.0)
    assert cdll.rbffd_solve(ctypes.byref(A), None, 0x4000, 0x5000, ctypes.byref(bad_tol), ctypes.byref(info),
                            0x6000, 1 << 30, None) == 1
    mixed = rbffd.make_opts(precision="mixed")
    # mixed precision without the float32 matrix
    assert cdll.rbffd_solve(ctypes.byref(A), None, 0x4000, 0x5000, ctypes.byref(mixed), ctypes.byref(info),
                            0x6000, 1 << 30, None) == 1
    ok = rbffd.make_opts()
    assert cdll.rbffd_solve(ctypes.byref(A), None, 0x4000, 0x5000, ctypes.byref(ok), ctypes.byref(info),
                            0x6000, 16, None) == 7
    A_wrong_dtype = rbffd.Csr(10, 30, 0x1000, 0x2000, 0x3000, 1)
    assert cdll.rbffd_solve(ctypes.byref(A_wrong_dtype), None, 0x4000, 0x5000, ctypes.byref(ok),
                            ctypes.byref(info), 0x6000, 1 << 30, None) == 1


def test_multigrid_argument_errors(cdll):
    """Multigrid entry points reject bad arguments before touching the device."""
    from paper_2107_03632_gb300 import rbffd

    INVALID, WS = 1, 7
    A = rbffd.Csr(1000, 12000, 0x1000, 0x2000, 0x3000, 0)
    A32_wrong_pattern = rbffd.Csr(1000, 12000, 0x1100, 0x2000, 0x4000, 1)
    h = rbffd.MgHandle()
    ws = cdll.rbffd_mg_workspace_size(1000, 12000)
    assert ws > 0 and cdll.rbffd_mg_workspace_size(0, 0) == 0
    args = dict(nu=2, omega=0.5)
    setup = lambda xy, N, a, a32, nu, om, w, nb: cdll.rbffd_mg_setup(  # noqa: E731
        xy, 0x5000, N, ctypes.byref(a) if a else None, ctypes.byref(a32) if a32 else None, nu, om,
        ctypes.byref(h), w, nb, None)
    assert setup(0x7000, 1000, A, None, 2, 0.5, 0x8000, ws - 1) == WS  # workspace too small
    assert setup(0x7000, 1000, A, None, 2, 0.5, 0x8001, ws) == WS  # misaligned workspace
    assert setup(0x7008, 1000, A, None, 2, 0.5, 0x8000, ws) == INVALID  # xy not 16-B aligned
    assert setup(0x7000, 999, A, None, 2, 0.5, 0x8000, ws) == INVALID  # N != rows of A
    assert setup(0x7000, 1000, None, None, 2, 0.5, 0x8000, ws) == INVALID
    assert setup(0x7000, 1000, A, A32_wrong_pattern, 2, 0.5, 0x8000, ws) == INVALID
    assert setup(0x7000, 1000, A, None, 0, 0.5, 0x8000, ws) == INVALID  # nu
    assert setup(0x7000, 1000, A, None, 2, 1.0, 0x8000, ws) == INVALID  # omega
    assert cdll.rbffd_mg_levels(ctypes.byref(h), None) == 0  # nothing built
    lv = rbffd.MgLevelInfo()
    assert cdll.rbffd_mg_level(ctypes.byref(h), 0, ctypes.byref(lv)) == INVALID
    assert cdll.rbffd_mg_level(None, 0, ctypes.byref(lv)) == INVALID
    assert cdll.rbffd_mg_apply(ctypes.byref(h), 0, 0x4000, 0x5000, None) == INVALID
    assert cdll.rbffd_mg_apply(None, 0, 0x4000, 0x5000, None) == INVALID
    # misfit gradient: argument errors before any launch
    assert cdll.rbffd_misfit_grad(None, 0x4000, 0x5000, 10, 0x6000, None) == INVALID
    assert cdll.rbffd_misfit_grad(0x3000, 0x4000, 0x5000, 0, 0x6000, None) == INVALID
    assert cdll.rbffd_misfit_grad(0x3000, 0x4000, None, 10, 0x6000, None) == INVALID
    h2 = rbffd.MgHandle()
    assert cdll.rbffd_mg_adjoint_of(ctypes.byref(h), ctypes.byref(A), None, ctypes.byref(h2), 0x8000, ws,
                                    None) == INVALID  # forward hierarchy never built
    assert cdll.rbffd_mg_adjoint_of(ctypes.byref(h), ctypes.byref(A), None, None, 0x8000, ws, None) == INVALID
    # a solve asking for multigrid with a handle that was never built
    opts = rbffd.make_opts()
    opts.precond = 1
    opts.mg = ctypes.pointer(h)
    info = rbffd.SolveInfo()
    assert cdll.rbffd_solve(ctypes.byref(A), None, 0x4000, 0x5000, ctypes.byref(opts), ctypes.byref(info),
                            0x6000, 1 << 30, None) == INVALID
    opts.precond = 2
    assert cdll.rbffd_solve(ctypes.byref(A), None, 0x4000, 0x5000, ctypes.byref(opts), ctypes.byref(info),
                            0x6000, 1 << 30, None) == INVALID
    # an adjoint solve with a hierarchy that was never built
    opts.precond = 1
    assert cdll.rbffd_solve_adjoint(ctypes.byref(A), None, 0x7000, 0x4000, 0x5000, None, None,
                                    ctypes.byref(opts), ctypes.byref(info), 0x6000, 1 << 30, None) == INVALID


def test_weights_config_table(cdll):
    """The weight-solve configuration table is host-side: pin, read back, reject, clear."""
    from paper_2107_03632_gb300 import rbffd

    c = rbffd.WeightsConfig()
    assert cdll.rbffd_weights_get_config(56, 6, ctypes.byref(c)) == 0
    assert (c.kernel, c.warps_per_block) == (2, 2)  # FP64 null-space, two warps, by default at m = 6
    assert cdll.rbffd_weights_get_config(30, 4, ctypes.byref(c)) == 0 and c.kernel == 7  # FP64, half a warp at m = 4
    assert cdll.rbffd_weights_get_config(90, 8, ctypes.byref(c)) == 0 and c.kernel == 2  # FP64, two warps, m = 8
    assert cdll.rbffd_weights_get_config(12, 0, ctypes.byref(c)) == 0 and c.kernel == 1  # m = 0: elimination
    pin = rbffd.WeightsConfig(1, 2, 0.0)
    assert cdll.rbffd_weights_set_config(30, 4, ctypes.byref(pin)) == 0
    assert cdll.rbffd_weights_get_config(30, 4, ctypes.byref(c)) == 0
    assert (c.kernel, c.warps_per_block) == (1, 2)
    assert cdll.rbffd_weights_set_config(30, 4, None) == 0
    assert cdll.rbffd_weights_get_config(30, 4, ctypes.byref(c)) == 0 and c.kernel == 7
    assert cdll.rbffd_weights_get_config(12, 2, ctypes.byref(c)) == 0 and c.kernel == 9  # FP64, a quarter warp
    for good in ((2, 2), (3, 4), (4, 1), (4, 3), (5, 2), (6, 4), (0, 2), (7, 1), (7, 4), (8, 2), (9, 1), (10, 4)):
        assert cdll.rbffd_weights_set_config(30, 4, ctypes.byref(rbffd.WeightsConfig(*good, 0.0))) == 0, good
    for bad in (rbffd.WeightsConfig(11, 1, 0.0), rbffd.WeightsConfig(3, 2, 0.0), rbffd.WeightsConfig(2, 1, 0.0),
                rbffd.WeightsConfig(9, 5, 0.0), rbffd.WeightsConfig(10, 0, 0.0),
                rbffd.WeightsConfig(7, 5, 0.0), rbffd.WeightsConfig(8, 0, 0.0),
                rbffd.WeightsConfig(5, 4, 0.0), rbffd.WeightsConfig(6, 2, 0.0), rbffd.WeightsConfig(4, 5, 0.0),
                rbffd.WeightsConfig(0, 5, 0.0),
                rbffd.WeightsConfig(0, 0, 0.0)):
        assert cdll.rbffd_weights_set_config(30, 4, ctypes.byref(bad)) == 1
    # double-float kernels only up to m = 6
    assert cdll.rbffd_weights_set_config(90, 8, ctypes.byref(rbffd.WeightsConfig(4, 1, 0.0))) == 1
    assert cdll.rbffd_weights_set_config(90, 8, ctypes.byref(rbffd.WeightsConfig(8, 1, 0.0))) == 1
    assert cdll.rbffd_weights_set_config(90, 8, ctypes.byref(rbffd.WeightsConfig(10, 1, 0.0))) == 1
    assert cdll.rbffd_weights_set_config(30, 4, None) == 0
    assert cdll.rbffd_weights_set_config(12, 0, ctypes.byref(rbffd.WeightsConfig(0, 1, 0.0))) == 1  # m = 0
    assert cdll.rbffd_weights_set_config(10, 4, ctypes.byref(pin)) == 1  # n < s
    assert cdll.rbffd_weights_autotune(None, 0x1000, 10, 6, 2, 0x2000, None, 0, None, None) == 1
    # an unknown precision selector is refused before any device access
    assert cdll.rbffd_weights_autotune(0x1000, 0x1000, 10, 6, 2, 0x2000, None, 7, None, None) == 1


# ------------------------------------------------------ bounds-checked build --
def test_normal_build_reports_no_checker(cdll):
    """The normal build has no violation records and reads back zeros."""
    from paper_2107_03632_gb300 import rbffd

    r = rbffd.rbffd_checked_read(reset=True)
    assert r == {"checked": 0, "violations": 0, "file": "", "line": 0, "index": 0, "bound": 0}


@pytest.mark.parametrize("args", [(8, 8, 0, 0, 0), (-1, 8, 0, 0, 0), (0, 8, 5, 4, 0), (0, 8, -1, 1, 0),
                                  (0, 8, 0, 0, 64), (0, 8, 0, 0, -8), (0, 8, 0, 0, 4), (0, 65, 0, 0, 0)])
def test_normal_build_refuses_out_of_range_probes(cdll, args):
    """The normal build's self-check entry takes in-range arguments only and
    refuses the rest on the host, before anything touches CUDA."""
    out = ctypes.c_void_p(0x1000)
    assert cdll.rbffd_checked_probe(*args, out, None) == 1  # RBFFD_ERR_INVALID_ARG


def test_checked_build_compiles_and_exports_every_symbol():
    """librbffd_checked.so (every computed index tested before its access)
    builds for sm_103a and exports the header's symbols; without a GPU its
    probe still refuses a bound above the table on the host."""
    from paper_2107_03632_gb300 import _build

    path = _build.build(checked=True)
    lib = ctypes.CDLL(path)
    names = declared_functions()
    for nm in names:
        assert hasattr(lib, nm), f"{nm} not exported by the checked build"
    f = lib.rbffd_checked_probe
    f.argtypes = [ctypes.c_int64] * 5 + [ctypes.c_void_p] * 2
    f.restype = ctypes.c_int
    assert f(0, 65, 0, 0, 0, ctypes.c_void_p(0x1000), None) == 1
