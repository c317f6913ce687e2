"""The RBF-FD Poisson pipeline on one GPU, composed from the C-ABI calls.

    stencils -> weights -> assemble (+ rhs) -> BiCGSTAB solve

plus a differentiable solve: `PoissonSolve.apply(f, g, op)` returns u with
A u = b(f, g); its backward runs the adjoint solve A^T lambda = dL/du and
maps lambda to dL/df (-lambda on interior rows) and dL/dg (+lambda on
Dirichlet rows), as b = -f inside and b = g on the boundary (Sec. IV,
Eqs. 2-3 at steady state).
"""

from __future__ import annotations

import torch

from . import rbffd as _r


class PoissonOperator:
    """Discrete Poisson operator on a node set (all tensors on one CUDA device)."""

    def __init__(self, xy: torch.Tensor, is_dirichlet: torch.Tensor, m: int, n: int, want_f32: bool = False):
        self.xy = xy
        self.is_dirichlet = is_dirichlet
        self.m, self.n = int(m), int(n)
        self.idx = _r.rbffd_stencils(xy, self.n)
        self.w, self.node_status = _r.rbffd_weights(xy, self.idx, self.m)
        self.A = _r.rbffd_assemble(self.idx, self.w, is_dirichlet, want_f32=want_f32)
        self._AT = None
        self._want_f32 = want_f32
        self._mg = None
        self._mga = None

    def check_stencils(self):
        bad = int(self.node_status.sum().item())
        if bad:
            raise _r.RbffdError(3, "rbffd_weights", f"{bad} singular stencil systems")

    @property
    def AT(self) -> _r.CsrMatrix:
        if self._AT is None:
            self._AT = _r.rbffd_transpose(self.A, want_f32=self._want_f32)
        return self._AT

    def multigrid(self) -> _r.Multigrid:
        """The multigrid hierarchy of A (built on first use)."""
        if self._mg is None:
            self._mg = _r.Multigrid(self.xy, self.is_dirichlet, self.A)
        return self._mg

    def multigrid_adjoint(self) -> _r.Multigrid:
        """The adjoint hierarchy, derived from the forward one."""
        if self._mga is None:
            self._mga = _r.Multigrid.adjoint_of(self.multigrid(), self.AT)
        return self._mga

    def rhs(self, f: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
        return _r.rbffd_rhs(f, g, self.is_dirichlet)

    def solve(self, b: torch.Tensor, x0: torch.Tensor | None = None, precond: str | None = None, **opts):
        """precond "mg": BiCGSTAB preconditioned by the multigrid V-cycle."""
        if precond == "mg":
            opts["mg"] = self.multigrid()
        return _r.rbffd_solve(self.A, b, x0, _r.make_opts(**opts))

    def solve_adjoint(self, dLdu: torch.Tensor, precond: str | None = None, **opts):
        if precond == "mg":
            opts["mg"] = self.multigrid_adjoint()
        return _r.rbffd_solve_adjoint(self.AT, self.is_dirichlet, dLdu, None, _r.make_opts(**opts))


def poisson_solve(xy, is_dirichlet, f, g, m: int, n: int, precision: str = "fp64", tol: float = 1e-10,
                  precond: str | None = None, **kw):
    """u solving the RBF-FD Poisson problem; returns (u, info, operator).
    precond "mg": multigrid-preconditioned BiCGSTAB."""
    op = PoissonOperator(xy, is_dirichlet, m, n, want_f32=(precision == "mixed"))
    op.check_stencils()
    b = op.rhs(f, g)
    u, info = op.solve(b, precision=precision, tol=tol, precond=precond, **kw)
    return u, info, op


class PoissonSolve(torch.autograd.Function):
    """u = A^{-1} b(f, g) with the adjoint gradient in backward."""

    # options that only make sense for the forward solve (its initial guess)
    _FORWARD_ONLY = ("x0",)

    @staticmethod
    def forward(ctx, f, g, op: PoissonOperator, opts: dict | None = None):
        opts = dict(opts or {})
        b = op.rhs(f.detach().contiguous(), g.detach().contiguous())
        u, info = op.solve(b, **opts)
        ctx.op = op
        ctx.opts = {k: v for k, v in opts.items() if k not in PoissonSolve._FORWARD_ONLY}
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, grad_u):
        need_f, need_g = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_f or need_g):
            return None, None, None, None
        lam, dLdf, dLdg, _ = ctx.op.solve_adjoint(grad_u.detach().contiguous(), **ctx.opts)
        return (dLdf if need_f else None), (dLdg if need_g else None), None, None
