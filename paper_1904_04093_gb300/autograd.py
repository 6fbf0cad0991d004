"""Differentiable GaBP solve: ``x = A^{-1} b`` with a hand-written adjoint.

The backward pass does not unroll sweeps.  At the solution, implicit
differentiation of ``A x = b`` gives, for an upstream gradient ``g = dL/dx``,

    dL/db = lam,  lam = A^{-T} g          (a GaBP solve on the transpose)
    dL/dA_ij = -lam_i x_j                  (on every stored entry)

Both run in the CUDA library (``gabp_solve_transpose``, ``gabp_edge_grad``).
The transpose has the same pattern and the same precision messages as A
(the diagonal corrections are symmetric in each edge pair), so the same
context serves both directions.  The paper has no counterpart: it solves
only forward problems.
"""
from __future__ import annotations

import torch

from . import GabpError, OK


class GabpSolveFunction(torch.autograd.Function):
    """``x = gabp_solve(values, b)`` for a fixed sparsity pattern held by ``solver``."""

    @staticmethod
    def forward(ctx, values, b, solver, tol, max_iter):
        # CUDA values stay on the device (gabp_set_values_device)
        solver.set_values(values.detach())
        x, it, rr, st = solver.solve(b.detach().contiguous(), tol, max_iter)
        if st != OK:
            raise GabpError(st, f"forward solve stopped with status {st} (rr={rr:.3e})")
        ctx.solver, ctx.tol, ctx.max_iter = solver, tol, max_iter
        ctx.values_device = values.device
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        solver = ctx.solver
        lam, it, rr, st = solver.solve_transpose(gx.detach().contiguous().double(), ctx.tol, ctx.max_iter)
        if st != OK:
            raise GabpError(st, f"adjoint solve stopped with status {st} (rr={rr:.3e})")
        dA = solver.edge_grad(lam, x)
        return dA.to(ctx.values_device), lam, None, None, None


def gabp_solve(values, b, solver, tol: float = 1e-12, max_iter: int = 200000):
    """Differentiable solve of ``A(values) x = b``; ``values`` follow the solver's CSR slots."""
    return GabpSolveFunction.apply(values, b, solver, tol, max_iter)
