"""Differentiable sparse solve x = A^-1 b through the adaptive s-step GMRES.

Forward: the library's solver.  Backward (adjoint method): the same solver on
A^T gives lam = A^-T dL/dx; then dL/db = lam and dL/dA_ij = -lam_i x_j on
A's pattern (the library's sampled outer product).  A is a fixed CSR pattern
analysed once by the Solver; its values are the differentiable input.
A^T has A's eigenvalues, so the adjoint solve takes the forward solve's
Ritz values as its shifts and skips its own pre-pass (reuse_ritz=False
runs it).
"""
from __future__ import annotations

import torch


class SparseSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, b, solver, opts):
        solver.update_values(values.detach())
        fopts = {k: v for k, v in opts.items() if k != "reuse_ritz"}
        x, info = solver.solve(b.detach().to(torch.float64), **fopts)
        if not info.converged:
            raise RuntimeError(f"forward solve did not converge "
                               f"(relres {info.final_relres:.3e})")
        ctx.solver, ctx.opts = solver, opts
        ctx.save_for_backward(x)
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, grad_x):
        (x,) = ctx.saved_tensors
        solver = ctx.solver
        opts = dict(ctx.opts)
        if opts.pop("reuse_ritz", True) and "ritz" not in opts:
            opts["ritz"] = ctx.info.ritz
        lam, info = solver.solve_adjoint(grad_x.contiguous().to(torch.float64),
                                         **opts)
        if not info.converged:
            raise RuntimeError(f"adjoint solve did not converge "
                               f"(relres {info.final_relres:.3e})")
        dval = solver.grad_values(lam, x)
        return dval, lam, None, None


def sparse_solve(values, b, solver, **opts):
    """x = A(values)^-1 b, differentiable in values and b."""
    return SparseSolve.apply(values, b, solver, opts)
