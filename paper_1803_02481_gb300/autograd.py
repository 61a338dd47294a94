"""Differentiable BoxMG solve (adjoint gradient).

``BoxMGSolve.apply(theta, b)`` returns u = A(exp(theta))^{-1} b.  Its
backward solves the adjoint equation A lambda = dL/du on the same hierarchy
(the diffusion operator is symmetric, so A^T = A) and applies the backward of
the finite-volume assembly (bmg_assemble_backward):

    dL/dtheta_c = -k_c sum_f dA_f/dk_c (u_c - u_n)(lambda_c - lambda_n)
                  - 2 k_c u_c lambda_c (per boundary face),    dL/db = lambda.

Everything numeric runs in the CUDA library; this module only orders the
calls and keeps the hierarchy alive between forward and backward.

The adjoint right-hand side dL/du is usually smooth, and A^{-1} amplifies a
smooth vector by up to ~n^2: its FP64 residual floor can sit above the
forward tolerance (about 1e-10 relative on a 2047^2 log-normal field).  The
adjoint solve therefore stops at ``adjoint_tol`` or after
``adjoint_max_cycles`` cycles, whichever comes first, and uses that iterate.

``solver``: "vcycle" (V(2,1) cycles, Algorithm 1) or "pcg" (CG
preconditioned by one symmetric V(1,1) cycle) for both solves; A is
symmetric, so the adjoint solve can use either on the same hierarchy.
"""
from __future__ import annotations

import torch

from . import BMG_FP64, BMG_SOLVER_PCG, default_options, setup


def _options(solver, max_cycles):
    if solver == "vcycle":
        return default_options(precision=BMG_FP64, log_coefficients=1, max_cycles=max_cycles)
    if solver == "pcg":
        return default_options(precision=BMG_FP64, log_coefficients=1, max_cycles=max_cycles,
                               nu1=1, nu2=1, solver=BMG_SOLVER_PCG)
    raise ValueError(f"solver must be 'vcycle' or 'pcg', got {solver!r}")


class BoxMGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, b, tol=1e-12, max_cycles=500, adjoint_tol=1e-12, adjoint_max_cycles=200,
                solver="vcycle"):
        opts = _options(solver, max_cycles)
        h = setup(theta.detach().contiguous(), opts)
        u, info = h.solve(b.detach().contiguous(), tol=tol)
        ctx.h = h
        ctx.adjoint = (adjoint_tol, adjoint_max_cycles)
        ctx.info = info
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        h = ctx.h
        atol, acyc = ctx.adjoint
        h.set_max_cycles(acyc)
        lam, info = h.solve(grad_u.contiguous(), tol=atol, allow_noconv=True)
        ctx.adjoint_info = info
        dtheta = torch.empty_like(u)
        h.assemble_backward(u, lam, dtheta)
        h.destroy()
        ctx.h = None
        return dtheta, lam, None, None, None, None, None


def solve(theta, b, tol=1e-12, max_cycles=500, adjoint_tol=1e-12, adjoint_max_cycles=200,
          solver="vcycle"):
    """u = A(exp(theta))^{-1} b, differentiable in theta and b; `solver`
    "vcycle" or "pcg" for the forward and the adjoint solve."""
    return BoxMGSolve.apply(theta, b, tol, max_cycles, adjoint_tol, adjoint_max_cycles, solver)
