"""Thin ctypes binding of librbffd (include/rbffd.h).

Argument marshalling only: every function here allocates the output tensors
and the workspace with torch on the input's device, passes raw device
pointers and the current CUDA stream to the C ABI, and raises on a non-OK
status.  All compute runs in the library's CUDA kernels; there is no CPU
fallback.  The function names are those of the C entry points.
"""

from __future__ import annotations

import ctypes
import dataclasses
import os

import torch

from . import _build

_LIB = None

RBFFD_OK = 0
STATUS_NAMES = {
    0: "RBFFD_OK",
    1: "RBFFD_ERR_INVALID_ARG",
    2: "RBFFD_ERR_CUDA",
    3: "RBFFD_ERR_SINGULAR_STENCIL",
    4: "RBFFD_ERR_NOT_CONVERGED",
    5: "RBFFD_ERR_BREAKDOWN",
    6: "RBFFD_ERR_TIMEOUT",
    7: "RBFFD_ERR_WORKSPACE",
}
for _code, _name in STATUS_NAMES.items():
    globals()[_name] = _code


class RbffdError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS_NAMES.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class Csr(ctypes.Structure):
    _fields_ = [
        ("n_rows", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("row_ptr", ctypes.c_void_p),
        ("col", ctypes.c_void_p),
        ("val", ctypes.c_void_p),
        ("dtype", ctypes.c_int32),
    ]


# rbffd_weights_config.kernel ids
WEIGHTS_KERNELS = ("null-space", "gauss", "null-space-2warp", "null-space-4warp", "null-space-df",
                   "null-space-df-2warp", "null-space-df-4warp", "null-space-half", "null-space-df-half",
                   "null-space-quarter", "null-space-df-quarter")


class WeightsConfig(ctypes.Structure):
    _fields_ = [
        ("kernel", ctypes.c_int32),
        ("warps_per_block", ctypes.c_int32),
        ("ms_per_mnode", ctypes.c_double),
    ]

    def as_dict(self):
        return {"kernel": WEIGHTS_KERNELS[self.kernel],
                "warps_per_block": self.warps_per_block, "ms_per_mnode": self.ms_per_mnode}


class MgHandle(ctypes.Structure):
    """rbffd_mg: host object filled by rbffd_mg_setup (opaque)."""

    _fields_ = [("opaque", ctypes.c_uint64 * 2048)]


MG_MAX_LEVELS = 24


class MgLevelInfo(ctypes.Structure):
    """rbffd_mg_level_info: device pointers into a built hierarchy."""

    _fields_ = [
        ("n_nodes", ctypes.c_int64),
        ("xy", ctypes.c_void_p),
        ("is_dirichlet", ctypes.c_void_p),
        ("A", Csr),
        ("w", ctypes.c_void_p),
        ("p_idx", ctypes.c_void_p),
        ("p_val", ctypes.c_void_p),
        ("p_k", ctypes.c_int32),
        ("minv", ctypes.c_void_p),
    ]


class _DeviceArray:
    """A raw device pointer seen as a torch tensor (__cuda_array_interface__);
    the memory stays owned by whoever allocated it."""

    _TYPESTR = {torch.float64: "<f8", torch.int64: "<i8", torch.int32: "<i4", torch.uint8: "|u1"}

    def __init__(self, ptr: int, shape: tuple, dtype: torch.dtype):
        self.__cuda_array_interface__ = {"shape": tuple(int(d) for d in shape), "typestr": self._TYPESTR[dtype],
                                         "data": (int(ptr), False), "version": 2, "strides": None}


def _device_copy(ptr: int, shape: tuple, dtype: torch.dtype, device: torch.device) -> torch.Tensor:
    with torch.cuda.device(device):
        return torch.as_tensor(_DeviceArray(ptr, shape, dtype), device=device).clone()


class SolveOpts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("inner_tol", ctypes.c_double),
        ("max_outer", ctypes.c_int32),
        ("jacobi", ctypes.c_int32),
        ("precond", ctypes.c_int32),
        ("mg", ctypes.POINTER(MgHandle)),
        ("spin_limit", ctypes.c_int64),
        ("wait_test", ctypes.c_int32),
        ("persistent", ctypes.c_int32),
        ("device_loop", ctypes.c_int32),
    ]


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("iters", ctypes.c_int32),
        ("outer_sweeps", ctypes.c_int32),
        ("restarts", ctypes.c_int32),
        ("rel_residual", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int64),
        ("spmv64_launches", ctypes.c_int64),
        ("spmv64_ms", ctypes.c_double),
        ("spmv64_bytes", ctypes.c_int64),
        ("spmv32_launches", ctypes.c_int64),
        ("spmv32_ms", ctypes.c_double),
        ("spmv32_bytes", ctypes.c_int64),
        ("mg_launches", ctypes.c_int64),
        ("mg_ms", ctypes.c_double),
        ("mg_bytes", ctypes.c_int64),
        ("batch_iter_launches", ctypes.c_int64),
        ("batch_iter_ms", ctypes.c_double),
        ("batch_iter_bytes", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CheckedReport(ctypes.Structure):
    _fields_ = [
        ("checked", ctypes.c_int32),
        ("line", ctypes.c_int32),
        ("file", ctypes.c_char * 32),
        ("violations", ctypes.c_int64),
        ("index", ctypes.c_int64),
        ("bound", ctypes.c_int64),
    ]


class BatchDesc(ctypes.Structure):
    _fields_ = [
        ("node_offset", ctypes.c_int64),
        ("n_nodes", ctypes.c_int64),
        ("m", ctypes.c_int32),
        ("n", ctypes.c_int32),
    ]


# (name, restype, argtypes) of every exported symbol declared in include/rbffd.h
_VP, _I64, _I32, _SZ, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t, ctypes.c_double
SIGNATURES = {
    "rbffd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rbffd_last_cuda_error": (ctypes.c_char_p, []),
    "rbffd_version": (ctypes.c_int, []),
    "rbffd_stencils_workspace_size": (_SZ, [_I64, _I32]),
    "rbffd_stencils": (ctypes.c_int, [_VP, _I64, _I32, _VP, _VP, _SZ, _VP]),
    "rbffd_stencils_noalloc": (ctypes.c_int, [_VP, _I64, _I32, _VP, _VP]),
    "rbffd_weights": (ctypes.c_int, [_VP, _VP, _I64, _I32, _I32, _VP, _VP, _VP]),
    "rbffd_weights_autotune": (ctypes.c_int, [_VP, _VP, _I64, _I32, _I32, _VP, _VP, _I32, ctypes.POINTER(WeightsConfig),
                                              _VP]),
    "rbffd_weights_get_config": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(WeightsConfig)]),
    "rbffd_weights_set_config": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(WeightsConfig)]),
    "rbffd_assemble_workspace_size": (_SZ, [_I64]),
    "rbffd_assemble_pattern": (ctypes.c_int, [_VP, _I64, _I32, _VP, _VP, _SZ, _VP]),
    "rbffd_assemble": (ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, _VP, _I64, _VP, _VP, _VP, _VP]),
    "rbffd_rhs": (ctypes.c_int, [_VP, _VP, _VP, _I64, _VP, _VP]),
    "rbffd_transpose_workspace_size": (_SZ, [_I64]),
    "rbffd_transpose": (ctypes.c_int, [ctypes.POINTER(Csr), _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "rbffd_solve_workspace_size": (_SZ, [_I64, ctypes.POINTER(SolveOpts)]),
    "rbffd_solve": (ctypes.c_int, [ctypes.POINTER(Csr), ctypes.POINTER(Csr), _VP, _VP,
                                   ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), _VP, _SZ, _VP]),
    "rbffd_solve_adjoint": (ctypes.c_int, [ctypes.POINTER(Csr), ctypes.POINTER(Csr), _VP, _VP, _VP, _VP, _VP,
                                           ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), _VP, _SZ, _VP]),
    "rbffd_misfit_grad": (ctypes.c_int, [_VP, _VP, _VP, _I64, _VP, _VP]),
    "rbffd_batched_workspace_size": (_SZ, [ctypes.POINTER(BatchDesc), _I32, _I32, ctypes.POINTER(SolveOpts)]),
    "rbffd_solve_batched": (ctypes.c_int, [ctypes.POINTER(BatchDesc), _I32, _VP, _VP, _VP, _VP, _I32, _VP,
                                           ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), _VP, _SZ, _VP]),
    "rbffd_explicit_workspace_size": (_SZ, [_I64, _I32]),
    "rbffd_explicit_pack": (ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, ctypes.POINTER(ctypes.c_int64), _VP, _SZ,
                                           _VP]),
    "rbffd_explicit_run": (ctypes.c_int, [_VP, _VP, _I64, _I32, _I64, _D, _I64, _VP, _SZ, _VP]),
    "rbffd_mg_workspace_size": (_SZ, [_I64, _I64]),
    "rbffd_mg_setup": (ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(Csr), ctypes.POINTER(Csr), _I32, _D,
                                      ctypes.POINTER(MgHandle), _VP, _SZ, _VP]),
    "rbffd_mg_setup_adjoint": (ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(Csr), ctypes.POINTER(Csr), _I32, _D,
                                              ctypes.POINTER(MgHandle), _VP, _SZ, _VP]),
    "rbffd_mg_setup_geometry": (ctypes.c_int, [_VP, _VP, _I64, _I32, _D, ctypes.POINTER(MgHandle), _VP, _SZ, _VP]),
    "rbffd_mg_setup_operator": (ctypes.c_int, [ctypes.POINTER(MgHandle), ctypes.POINTER(Csr), ctypes.POINTER(Csr),
                                               _VP]),
    "rbffd_mg_levels": (ctypes.c_int, [ctypes.POINTER(MgHandle), ctypes.POINTER(ctypes.c_int64)]),
    "rbffd_mg_level": (ctypes.c_int, [ctypes.POINTER(MgHandle), ctypes.c_int32, ctypes.POINTER(MgLevelInfo)]),
    "rbffd_mg_adjoint_of": (ctypes.c_int, [ctypes.POINTER(MgHandle), ctypes.POINTER(Csr), ctypes.POINTER(Csr),
                                           ctypes.POINTER(MgHandle), ctypes.c_void_p, ctypes.c_size_t,
                                           ctypes.c_void_p]),
    "rbffd_mg_galerkin_workspace_size": (_SZ, [ctypes.POINTER(MgHandle)]),
    "rbffd_mg_galerkin_adjoint": (ctypes.c_int, [ctypes.POINTER(MgHandle), ctypes.POINTER(Csr), ctypes.POINTER(Csr),
                                                 ctypes.POINTER(MgHandle), ctypes.c_void_p, ctypes.c_size_t,
                                                 ctypes.c_void_p]),
    "rbffd_mg_apply": (ctypes.c_int, [ctypes.POINTER(MgHandle), ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "rbffd_diag_recip": (ctypes.c_int, [_VP, _I64, _VP, _VP, _VP]),
    "rbffd_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "rbffd_profile_read": (ctypes.c_int, [ctypes.POINTER(Profile), ctypes.c_int]),
    "rbffd_checked_read": (ctypes.c_int, [ctypes.POINTER(CheckedReport), ctypes.c_int]),
    "rbffd_checked_probe": (ctypes.c_int, [_I64, _I64, _I64, _I64, _I64, _VP, _VP]),
}


def checked_build_selected() -> bool:
    """RBFFD_CHECKED=1 in the environment selects the bounds-checked library."""
    return os.environ.get("RBFFD_CHECKED", "0") == "1"


def lib_path() -> str:
    return _build.lib_path(checked_build_selected())


def load(build_if_missing: bool = True):
    """Load librbffd.so, or librbffd_checked.so under RBFFD_CHECKED=1
    (building it when missing); raises if it cannot be loaded."""
    global _LIB
    if _LIB is not None:
        return _LIB
    checked = checked_build_selected()
    path = _build.lib_path(checked)
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"librbffd not built at {path}")
        _build.build(checked=checked)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status: int, where: str):
    if status != RBFFD_OK:
        detail = ""
        if status == 2:
            detail = load().rbffd_last_cuda_error().decode()
        raise RbffdError(status, where, detail)


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _ptr(t) -> int:
    return 0 if t is None else t.data_ptr()


def _require(t, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def _workspace(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


# ----------------------------------------------------------------- stencils --
def rbffd_stencils(xy: torch.Tensor, n: int, idx: torch.Tensor | None = None,
                   ws: torch.Tensor | None = None) -> torch.Tensor:
    _require(xy, torch.float64, "xy")
    N = xy.shape[0]
    if xy.dim() != 2 or xy.shape[1] != 2:
        raise ValueError("xy must be N x 2")
    lib = load()
    if idx is None:
        idx = torch.empty((N, n), dtype=torch.int32, device=xy.device)
    _require(idx, torch.int32, "idx", (N, n))
    if ws is None:
        ws = _workspace(lib.rbffd_stencils_workspace_size(N, n), xy.device)
    _check(lib.rbffd_stencils(_ptr(xy), N, n, _ptr(idx), _ptr(ws), ws.numel(), _stream(xy.device)),
           "rbffd_stencils")
    return idx


def rbffd_weights(xy: torch.Tensor, idx: torch.Tensor, m: int, w: torch.Tensor | None = None,
                  node_status: torch.Tensor | None = None, want_status: bool = True):
    _require(xy, torch.float64, "xy")
    _require(idx, torch.int32, "idx")
    N, n = idx.shape
    lib = load()
    if w is None:
        w = torch.empty((N, n), dtype=torch.float64, device=xy.device)
    if node_status is None and want_status:
        node_status = torch.empty(N, dtype=torch.int32, device=xy.device)
    _require(w, torch.float64, "w", (N, n))
    _check(lib.rbffd_weights(_ptr(xy), _ptr(idx), N, n, m, _ptr(w), _ptr(node_status), _stream(xy.device)),
           "rbffd_weights")
    return w, node_status


# ----------------------------------------------------------------- assembly --
@dataclasses.dataclass
class CsrMatrix:
    """CSR matrix held in torch tensors (row_ptr int64, col int32, val f64, optional val32)."""

    row_ptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor
    val32: torch.Tensor | None = None

    @property
    def n_rows(self) -> int:
        return self.row_ptr.numel() - 1

    @property
    def nnz(self) -> int:
        return self.col.numel()

    def c64(self) -> Csr:
        return Csr(self.n_rows, self.nnz, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val), 0)

    def c32(self) -> Csr | None:
        if self.val32 is None:
            return None
        return Csr(self.n_rows, self.nnz, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val32), 1)


def rbffd_assemble_pattern(is_dirichlet: torch.Tensor, n: int, row_ptr: torch.Tensor | None = None,
                           ws: torch.Tensor | None = None) -> torch.Tensor:
    _require(is_dirichlet, torch.uint8, "is_dirichlet")
    N = is_dirichlet.numel()
    lib = load()
    if row_ptr is None:
        row_ptr = torch.empty(N + 1, dtype=torch.int64, device=is_dirichlet.device)
    _require(row_ptr, torch.int64, "row_ptr", (N + 1,))
    if ws is None:
        ws = _workspace(lib.rbffd_assemble_workspace_size(N), is_dirichlet.device)
    _check(lib.rbffd_assemble_pattern(_ptr(is_dirichlet), N, n, _ptr(row_ptr), _ptr(ws), ws.numel(),
                                      _stream(is_dirichlet.device)), "rbffd_assemble_pattern")
    return row_ptr


def rbffd_assemble(idx: torch.Tensor, w: torch.Tensor, is_dirichlet: torch.Tensor,
                   row_ptr: torch.Tensor | None = None, nnz: int | None = None,
                   want_f32: bool = False, out: CsrMatrix | None = None) -> CsrMatrix:
    """CSR of the Poisson operator.  With `out`, its row_ptr (already holding
    the pattern) and col/val(/val32) buffers are filled in place, without a
    device->host read."""
    _require(idx, torch.int32, "idx")
    N, n = idx.shape
    _require(w, torch.float64, "w", (N, n))
    _require(is_dirichlet, torch.uint8, "is_dirichlet", (N,))
    lib = load()
    dev = idx.device
    if out is not None:
        row_ptr, col, val, val32 = out.row_ptr, out.col, out.val, out.val32
        nnz = col.numel()
        _require(row_ptr, torch.int64, "row_ptr", (N + 1,))
        _require(val, torch.float64, "val", (nnz,))
        if val32 is not None:
            _require(val32, torch.float32, "val32", (nnz,))
    else:
        if row_ptr is None:
            row_ptr = rbffd_assemble_pattern(is_dirichlet, n)
        if nnz is None:
            nnz = int(row_ptr[-1].item())  # one device->host read to size col/val
        col = torch.empty(nnz, dtype=torch.int32, device=dev)
        val = torch.empty(nnz, dtype=torch.float64, device=dev)
        val32 = torch.empty(nnz, dtype=torch.float32, device=dev) if want_f32 else None
    _check(lib.rbffd_assemble(_ptr(idx), _ptr(w), _ptr(is_dirichlet), N, n, _ptr(row_ptr), nnz, _ptr(col),
                              _ptr(val), _ptr(val32), _stream(dev)), "rbffd_assemble")
    return CsrMatrix(row_ptr, col, val, val32)


def rbffd_rhs(f: torch.Tensor, g: torch.Tensor, is_dirichlet: torch.Tensor, b: torch.Tensor | None = None):
    _require(f, torch.float64, "f")
    N = f.numel()
    _require(g, torch.float64, "g", (N,))
    _require(is_dirichlet, torch.uint8, "is_dirichlet", (N,))
    lib = load()
    if b is None:
        b = torch.empty(N, dtype=torch.float64, device=f.device)
    _check(lib.rbffd_rhs(_ptr(f), _ptr(g), _ptr(is_dirichlet), N, _ptr(b), _stream(f.device)), "rbffd_rhs")
    return b


def rbffd_transpose(A: CsrMatrix, want_f32: bool = False) -> CsrMatrix:
    lib = load()
    dev = A.val.device
    N, nnz = A.n_rows, A.nnz
    row_ptr_t = torch.empty(N + 1, dtype=torch.int64, device=dev)
    col_t = torch.empty(nnz, dtype=torch.int32, device=dev)
    val_t = torch.empty(nnz, dtype=torch.float64, device=dev)
    val32 = torch.empty(nnz, dtype=torch.float32, device=dev) if want_f32 else None
    ws = _workspace(lib.rbffd_transpose_workspace_size(N), dev)
    c = A.c64()
    _check(lib.rbffd_transpose(ctypes.byref(c), _ptr(row_ptr_t), _ptr(col_t), _ptr(val_t),
                               _ptr(val32) if val32 is not None else None, _ptr(ws), ws.numel(), _stream(dev)),
           "rbffd_transpose")
    return CsrMatrix(row_ptr_t, col_t, val_t, val32)


# -------------------------------------------------------------------- solve --
def make_opts(tol=1e-10, max_iter=200000, precision="fp64", inner_tol=None, max_outer=1000, jacobi=True,
              mg: "Multigrid | None" = None):
    """Solver options.  inner_tol: residual reduction per restarted pass
    (default 1e-3 for FP64, 1e-5 for mixed; 1e-10 with multigrid, i.e. one
    pass).  mg: a Multigrid hierarchy -> BiCGSTAB right-preconditioned by its
    V-cycle (float32 V-cycle when precision is "mixed")."""
    prec = {"fp64": 0, "mixed": 1}[precision]
    if inner_tol is None:
        inner_tol = 1e-10 if mg is not None else (1e-5 if prec == 1 else 1e-3)
    o = SolveOpts(float(tol), int(max_iter), prec, float(inner_tol), int(max_outer), 1 if jacobi else 0, 0, None,
                  0, 0, 0, 0)
    if mg is not None:
        o.precond = 1
        o.mg = ctypes.pointer(mg.handle)
        o._mg_ref = mg  # keeps the hierarchy (and its device workspace) alive
    return o


class Multigrid:
    """Geometric multigrid hierarchy for the operator A of a node set (rbffd_mg_setup).

    Holds the host handle and the device workspace it points into."""

    def __init__(self, xy: torch.Tensor, is_dirichlet: torch.Tensor, A: "CsrMatrix", nu: int = 2,
                 omega: float = 0.6, ws: torch.Tensor | None = None, adjoint: bool = False):
        """adjoint=True: A is A^T (the adjoint solve's matrix) and the hierarchy
        is the transposed one (rbffd_mg_setup_adjoint)."""
        N = xy.shape[0]
        _require(xy, torch.float64, "xy", (N, 2))
        _require(is_dirichlet, torch.uint8, "is_dirichlet", (N,))
        self.handle = MgHandle()
        if ws is None:
            ws = mg_workspace(N, A.nnz, xy.device)
        self.ws = ws
        self.adjoint = adjoint
        self.galerkin = False
        self.setup(xy, is_dirichlet, A, nu, omega)

    def setup(self, xy: torch.Tensor, is_dirichlet: torch.Tensor, A: "CsrMatrix", nu: int = 2, omega: float = 0.6):
        """(Re)builds the hierarchy in the same workspace (same node count)."""
        lib = load()
        c64 = A.c64()
        c32 = A.c32()
        self.A = A
        fn = lib.rbffd_mg_setup_adjoint if self.adjoint else lib.rbffd_mg_setup
        _check(fn(_ptr(xy), _ptr(is_dirichlet), xy.shape[0], ctypes.byref(c64),
                  ctypes.byref(c32) if c32 is not None else None, int(nu), float(omega),
                  ctypes.byref(self.handle), _ptr(self.ws), self.ws.numel(), _stream(xy.device)),
               "rbffd_mg_setup_adjoint" if self.adjoint else "rbffd_mg_setup")

    def setup_geometry(self, xy: torch.Tensor, is_dirichlet: torch.Tensor, nu: int = 2, omega: float = 0.6,
                       stream: torch.cuda.Stream | None = None):
        """First phase of a rebuild (rbffd_mg_setup_geometry): everything that
        depends on the nodes and the mask only, on `stream` (default: the
        current one), which it synchronises.  A forward hierarchy only."""
        if self.adjoint:
            raise RbffdError(1, "rbffd_mg_setup_geometry", "forward hierarchies only")
        st = (stream or torch.cuda.current_stream(xy.device)).cuda_stream
        _check(load().rbffd_mg_setup_geometry(_ptr(xy), _ptr(is_dirichlet), xy.shape[0], int(nu), float(omega),
                                              ctypes.byref(self.handle), _ptr(self.ws), self.ws.numel(), st),
               "rbffd_mg_setup_geometry")

    def setup_operator(self, A: "CsrMatrix"):
        """Second phase (rbffd_mg_setup_operator): the fine operator A attached
        to level 0, on the current stream."""
        c64 = A.c64()
        c32 = A.c32()
        self.A = A
        _check(load().rbffd_mg_setup_operator(ctypes.byref(self.handle), ctypes.byref(c64),
                                              ctypes.byref(c32) if c32 is not None else None,
                                              _stream(A.val.device)), "rbffd_mg_setup_operator")

    @classmethod
    def adjoint_of(cls, fwd: "Multigrid", AT: "CsrMatrix", ws: torch.Tensor | None = None) -> "Multigrid":
        """The adjoint hierarchy of the built forward hierarchy fwd, for AT = A^T
        (rbffd_mg_adjoint_of: fwd's coarse levels reused, operators transposed)."""
        self = cls.__new__(cls)
        self.handle = MgHandle()
        self.ws = ws if ws is not None else mg_workspace(AT.n_rows, AT.nnz, AT.val.device)
        self.adjoint = True
        self.galerkin = False
        self.rebuild_from(fwd, AT)
        return self

    @classmethod
    def galerkin_adjoint_of(cls, fwd: "Multigrid", AT: "CsrMatrix", ws: torch.Tensor | None = None) -> "Multigrid":
        """The adjoint hierarchy of fwd with Galerkin coarse operators R A P
        (rbffd_mg_galerkin_adjoint); rbffd_solve_adjoint runs it
        right-preconditioned."""
        self = cls.__new__(cls)
        self.handle = MgHandle()
        if ws is None:
            nbytes = load().rbffd_mg_galerkin_workspace_size(ctypes.byref(fwd.handle))
            if nbytes == 0:
                raise RbffdError(1, "rbffd_mg_galerkin_workspace_size")
            ws = _workspace(nbytes, AT.val.device)
        self.ws = ws
        self.adjoint = True
        self.galerkin = True
        self.rebuild_from(fwd, AT)
        return self

    def rebuild_from(self, fwd: "Multigrid", AT: "CsrMatrix"):
        """(Re)builds this adjoint hierarchy from fwd (rbffd_mg_adjoint_of, or
        rbffd_mg_galerkin_adjoint for a Galerkin hierarchy)."""
        c64, c32 = AT.c64(), AT.c32()
        self.A = AT
        name = "rbffd_mg_galerkin_adjoint" if getattr(self, "galerkin", False) else "rbffd_mg_adjoint_of"
        _check(getattr(load(), name)(ctypes.byref(fwd.handle), ctypes.byref(c64),
                                     ctypes.byref(c32) if c32 is not None else None, ctypes.byref(self.handle),
                                     _ptr(self.ws), self.ws.numel(), _stream(AT.val.device)), name)

    def levels(self) -> list:
        arr = (ctypes.c_int64 * MG_MAX_LEVELS)()
        n = load().rbffd_mg_levels(ctypes.byref(self.handle), arr)
        return [int(arr[i]) for i in range(n)]

    def apply(self, b: torch.Tensor, out: torch.Tensor | None = None, fp32: bool = False) -> torch.Tensor:
        """out = M b, one preconditioner application (rbffd_mg_apply)."""
        N = self.levels()[0]
        _require(b, torch.float64, "b", (N,))
        if out is None:
            out = torch.empty_like(b)
        _require(out, torch.float64, "out", (N,))
        _check(load().rbffd_mg_apply(ctypes.byref(self.handle), 1 if fp32 else 0, _ptr(b), _ptr(out),
                                     _stream(b.device)), "rbffd_mg_apply")
        return out

    def level(self, level: int) -> dict:
        """Copies of one level's arrays (rbffd_mg_level): xy, is_dirichlet, the
        operator A (CsrMatrix), smoother weights w, prolongation p_idx/p_val
        into this level (None at the coarsest) and minv (coarsest only)."""
        info = MgLevelInfo()
        _check(load().rbffd_mg_level(ctypes.byref(self.handle), int(level), ctypes.byref(info)), "rbffd_mg_level")
        dev = self.ws.device
        n, nnz = info.n_nodes, info.A.nnz
        out = {
            "n_nodes": n,
            "xy": _device_copy(info.xy, (n, 2), torch.float64, dev),
            "is_dirichlet": _device_copy(info.is_dirichlet, (n,), torch.uint8, dev),
            "A": CsrMatrix(_device_copy(info.A.row_ptr, (n + 1,), torch.int64, dev),
                           _device_copy(info.A.col, (nnz,), torch.int32, dev),
                           _device_copy(info.A.val, (nnz,), torch.float64, dev)),
            "w": _device_copy(info.w, (n,), torch.float64, dev),
            "p_idx": None, "p_val": None, "minv": None,
        }
        if info.p_k:
            out["p_idx"] = _device_copy(info.p_idx, (n, info.p_k), torch.int32, dev)
            out["p_val"] = _device_copy(info.p_val, (n, info.p_k), torch.float64, dev)
        if info.minv:
            out["minv"] = _device_copy(info.minv, (n, n), torch.float64, dev)
        return out


class ExplicitLoop:
    """The explicit time loop of Eq. 4 on packed interior rows (rbffd_explicit_*)."""

    def __init__(self, idx: torch.Tensor, w: torch.Tensor, is_dirichlet: torch.Tensor, ws: torch.Tensor | None = None):
        N, n = idx.shape
        _require(idx, torch.int32, "idx", (N, n))
        _require(w, torch.float64, "w", (N, n))
        _require(is_dirichlet, torch.uint8, "is_dirichlet", (N,))
        lib = load()
        self.N, self.n = N, n
        self.ws = ws if ws is not None else _workspace(lib.rbffd_explicit_workspace_size(N, n), idx.device)
        ni = ctypes.c_int64(0)
        _check(lib.rbffd_explicit_pack(_ptr(idx), _ptr(w), _ptr(is_dirichlet), N, n, ctypes.byref(ni), _ptr(self.ws),
                                       self.ws.numel(), _stream(idx.device)), "rbffd_explicit_pack")
        self.n_interior = int(ni.value)

    def run(self, f: torch.Tensor, u: torch.Tensor, dt: float, steps: int) -> torch.Tensor:
        """Advances u in place by `steps` forward-Euler steps; returns u."""
        _require(f, torch.float64, "f", (self.N,))
        _require(u, torch.float64, "u", (self.N,))
        _check(load().rbffd_explicit_run(_ptr(f), _ptr(u), self.N, self.n, self.n_interior, float(dt), int(steps),
                                         _ptr(self.ws), self.ws.numel(), _stream(u.device)), "rbffd_explicit_run")
        return u


WEIGHTS_PRECISION = {"fp64": 0, "df": 1, "any": 2}  # RBFFD_WEIGHTS_FP64 / _DF / _ANY


def rbffd_weights_autotune(xy: torch.Tensor, idx: torch.Tensor, m: int, precision: str = "fp64") -> dict:
    """Times the weight-solve configurations of the given arithmetic ("fp64",
    "df" = double-float, "any") on (a sample of) these stencils and keeps the
    fastest for (n, m); returns it."""
    N, n = idx.shape
    _require(xy, torch.float64, "xy", (N, 2))
    _require(idx, torch.int32, "idx", (N, n))
    w = torch.empty((N, n), dtype=torch.float64, device=xy.device)
    st = torch.empty(N, dtype=torch.int32, device=xy.device)
    best = WeightsConfig()
    _check(load().rbffd_weights_autotune(_ptr(xy), _ptr(idx), N, n, int(m), _ptr(w), _ptr(st),
                                         WEIGHTS_PRECISION[precision], ctypes.byref(best), _stream(xy.device)),
           "rbffd_weights_autotune")
    return best.as_dict()


def weights_config(n: int, m: int) -> dict:
    c = WeightsConfig()
    _check(load().rbffd_weights_get_config(int(n), int(m), ctypes.byref(c)), "rbffd_weights_get_config")
    return c.as_dict()


def set_weights_config(n: int, m: int, kernel: str | None = None, warps_per_block: int = 0):
    """Pins the weight-solve configuration for (n, m); kernel None: back to the default."""
    lib = load()
    if kernel is None:
        _check(lib.rbffd_weights_set_config(int(n), int(m), None), "rbffd_weights_set_config")
        return
    c = WeightsConfig(WEIGHTS_KERNELS.index(kernel), int(warps_per_block), 0.0)
    _check(lib.rbffd_weights_set_config(int(n), int(m), ctypes.byref(c)), "rbffd_weights_set_config")


def mg_workspace(N: int, nnz: int, device) -> torch.Tensor:
    nbytes = load().rbffd_mg_workspace_size(N, nnz)
    if nbytes == 0:
        raise RbffdError(1, "rbffd_mg_workspace_size")
    return _workspace(nbytes, device)


def stencils_workspace(N: int, n: int, device) -> torch.Tensor:
    return _workspace(load().rbffd_stencils_workspace_size(N, n), device)


def assemble_workspace(N: int, device) -> torch.Tensor:
    return _workspace(load().rbffd_assemble_workspace_size(N), device)


def solve_workspace(N: int, opts: SolveOpts, device) -> torch.Tensor:
    return _workspace(load().rbffd_solve_workspace_size(N, ctypes.byref(opts)), device)


def rbffd_solve(A: CsrMatrix, b: torch.Tensor, x: torch.Tensor | None = None, opts: SolveOpts | None = None,
                ws: torch.Tensor | None = None, raise_on_error: bool = True):
    """Solve A x = b in place on x (zero initial guess when x is None); returns (x, info dict)."""
    _require(b, torch.float64, "b", (A.n_rows,))
    lib = load()
    opts = opts or make_opts()
    if x is None:
        x = torch.zeros_like(b)
    _require(x, torch.float64, "x", (A.n_rows,))
    if opts.precision == 1 and opts.precond == 0 and A.val32 is None:
        raise ValueError("mixed precision needs the float32 matrix copy (assemble with want_f32=True)")
    if ws is None:
        ws = solve_workspace(A.n_rows, opts, b.device)
    info = SolveInfo()
    c64 = A.c64()
    c32 = A.c32()
    st = lib.rbffd_solve(ctypes.byref(c64), ctypes.byref(c32) if c32 is not None else None, _ptr(b), _ptr(x),
                         ctypes.byref(opts), ctypes.byref(info), _ptr(ws), ws.numel(), _stream(b.device))
    if raise_on_error and st not in (RBFFD_OK,):
        _check(st, "rbffd_solve")
    d = info.as_dict()
    d["status_code"] = st
    return x, d


def rbffd_solve_adjoint(AT: CsrMatrix, is_dirichlet: torch.Tensor, dLdu: torch.Tensor,
                        lam: torch.Tensor | None = None, opts: SolveOpts | None = None,
                        ws: torch.Tensor | None = None, raise_on_error: bool = True):
    """lambda with A^T lambda = dL/du, and (dL/df, dL/dg); returns (lam, dLdf, dLdg, info dict)."""
    _require(dLdu, torch.float64, "dLdu", (AT.n_rows,))
    _require(is_dirichlet, torch.uint8, "is_dirichlet", (AT.n_rows,))
    lib = load()
    opts = opts or make_opts()
    if lam is None:
        lam = torch.zeros_like(dLdu)
    dLdf = torch.empty_like(dLdu)
    dLdg = torch.empty_like(dLdu)
    if ws is None:
        ws = solve_workspace(AT.n_rows, opts, dLdu.device)
    info = SolveInfo()
    c64 = AT.c64()
    c32 = AT.c32()
    st = lib.rbffd_solve_adjoint(ctypes.byref(c64), ctypes.byref(c32) if c32 is not None else None,
                                 _ptr(is_dirichlet), _ptr(dLdu), _ptr(lam), _ptr(dLdf), _ptr(dLdg),
                                 ctypes.byref(opts), ctypes.byref(info), _ptr(ws), ws.numel(), _stream(dLdu.device))
    if raise_on_error and st != RBFFD_OK:
        _check(st, "rbffd_solve_adjoint")
    d = info.as_dict()
    d["status_code"] = st
    return lam, dLdf, dLdg, d


def rbffd_misfit_grad(u: torch.Tensor, u_target: torch.Tensor, is_dirichlet: torch.Tensor,
                      out: torch.Tensor | None = None) -> torch.Tensor:
    """dL/du of L = sum_interior (u - u_target)^2."""
    N = u.shape[0]
    _require(u, torch.float64, "u", (N,))
    _require(u_target, torch.float64, "u_target", (N,))
    _require(is_dirichlet, torch.uint8, "is_dirichlet", (N,))
    if out is None:
        out = torch.empty_like(u)
    _check(load().rbffd_misfit_grad(_ptr(u), _ptr(u_target), _ptr(is_dirichlet), N, _ptr(out), _stream(u.device)),
           "rbffd_misfit_grad")
    return out


# --------------------------------------------------------------- profiling --
def rbffd_profile_enable(on: bool = True):
    _check(load().rbffd_profile_enable(1 if on else 0), "rbffd_profile_enable")


def rbffd_profile_read(reset: bool = False) -> dict:
    p = Profile()
    _check(load().rbffd_profile_read(ctypes.byref(p), 1 if reset else 0), "rbffd_profile_read")
    return p.as_dict()


def rbffd_checked_probe(index: int, bound: int, span_off: int = 0, span_len: int = 0, smem_off: int = 0,
                        device="cuda") -> torch.Tensor:
    """One self-check access of the bounds-checked build (see the header);
    returns the value read back (a 1-element device tensor)."""
    out = torch.zeros(1, dtype=torch.float64, device=device)
    _check(load().rbffd_checked_probe(int(index), int(bound), int(span_off), int(span_len), int(smem_off),
                                      _ptr(out), _stream(out.device)), "rbffd_checked_probe")
    return out


def rbffd_checked_read(reset: bool = False) -> dict:
    """Violation records of the bounds-checked build (checked = 0 and no
    violations in the normal build); synchronise the device first."""
    r = CheckedReport()
    _check(load().rbffd_checked_read(ctypes.byref(r), 1 if reset else 0), "rbffd_checked_read")
    return {"checked": int(r.checked), "violations": int(r.violations), "file": r.file.decode(),
            "line": int(r.line), "index": int(r.index), "bound": int(r.bound)}


# ----------------------------------------------------------------- batched --
def batch_descs(sizes):
    """Descriptor array for instances [(n_nodes, m, n), ...] stored back to back."""
    arr = (BatchDesc * len(sizes))()
    off = 0
    for i, (N, m, n) in enumerate(sizes):
        arr[i] = BatchDesc(off, int(N), int(m), int(n))
        off += int(N)
    return arr, off


def batched_workspace(sizes, n_rhs: int, device, opts: SolveOpts | None = None) -> torch.Tensor:
    descs, _ = batch_descs(sizes)
    nbytes = load().rbffd_batched_workspace_size(descs, len(sizes), n_rhs,
                                                 ctypes.byref(opts) if opts is not None else None)
    if nbytes == 0:
        raise RbffdError(1, "rbffd_batched_workspace_size")
    return _workspace(nbytes, device)


def rbffd_solve_batched(sizes, xy: torch.Tensor, is_dirichlet: torch.Tensor, f: torch.Tensor, g: torch.Tensor,
                        u: torch.Tensor | None = None, opts: SolveOpts | None = None, raise_on_error: bool = True,
                        ws: torch.Tensor | None = None):
    """Solve every instance for every right-hand side.  f, g, u: N_total x n_rhs
    (node-major); u holds the initial guess on entry.  Returns (u, list of
    per-instance info dicts, status)."""
    descs, N = batch_descs(sizes)
    _require(xy, torch.float64, "xy", (N, 2))
    _require(is_dirichlet, torch.uint8, "is_dirichlet", (N,))
    R = f.shape[1]
    _require(f, torch.float64, "f", (N, R))
    _require(g, torch.float64, "g", (N, R))
    lib = load()
    opts = opts or make_opts(precision="mixed")
    if u is None:
        u = torch.zeros_like(f)
    _require(u, torch.float64, "u", (N, R))
    if ws is None:
        ws = batched_workspace(sizes, R, xy.device, opts)
    infos = (SolveInfo * len(sizes))()
    st = lib.rbffd_solve_batched(descs, len(sizes), _ptr(xy), _ptr(is_dirichlet), _ptr(f), _ptr(g), R, _ptr(u),
                                 ctypes.byref(opts), infos, _ptr(ws), ws.numel(), _stream(xy.device))
    if raise_on_error and st != RBFFD_OK:
        _check(st, "rbffd_solve_batched")
    return u, [infos[i].as_dict() for i in range(len(sizes))], st
