"""torch.autograd.Function wrappers of libhq's differentiation entry points.

The forward passes run Algorithm 1 on an FP64 ``hq.Solver`` for the given
potential (warm-started from the solver's current block) and read the
Rayleigh-Ritz eigenpairs; the backward passes call hq_grad_eigs /
hq_grad_density.  Marshalling only: every step runs in libhq's kernels.

    lam_sum = EigenvalueSum.apply(V, solver, 1e-10, 20000)
    rho = Density.apply(V, solver, 1e-10, 20000)
    loss = 0.5 * h**3 * ((rho - rho_target) ** 2).sum()
    loss.backward()          # V.grad = dL/dV by the adjoint solves
"""
from __future__ import annotations

import numpy as np
import torch

from . import hq


def _solve_for(V, solver, eps, max_steps):
    Vd = V.detach().to(torch.float64).contiguous()
    solver.set_potential(Vd if Vd.is_cuda else Vd.numpy())
    solver.solve(eps, max_steps)


class EigenvalueSum(torch.autograd.Function):
    """sum_i w_i lambda_i(V) over the N lowest eigenvalues of -Delta_h/2 + V
    (w = None: all ones)."""

    @staticmethod
    def forward(ctx, V, solver, eps, max_steps, w=None):
        _solve_for(V, solver, eps, max_steps)
        lam = solver.eigenpairs()["lam_rr"]
        wn = None if w is None else np.asarray(w, dtype=np.float64)
        ctx.solver, ctx.w, ctx.device = solver, wn, V.device
        val = float(np.sum(lam if wn is None else wn * lam))
        return torch.tensor(val, dtype=torch.float64, device=V.device)

    @staticmethod
    def backward(ctx, grad):
        dV = torch.from_numpy(ctx.solver.grad_eigs(ctx.w)).to(ctx.device)
        return grad * dV, None, None, None, None


class Density(torch.autograd.Function):
    """rho(V) = sum_i u_i^2 over the N lowest eigenvectors (<u_i,u_i> = 1)."""

    @staticmethod
    def forward(ctx, V, solver, eps, max_steps, rtol=1e-10, maxit=500):
        _solve_for(V, solver, eps, max_steps)
        solver.eigenpairs()
        rho = solver.density()
        ctx.solver, ctx.device, ctx.rtol, ctx.maxit = solver, V.device, rtol, maxit
        return torch.from_numpy(rho).to(V.device)

    @staticmethod
    def backward(ctx, grad_rho):
        G = grad_rho.detach().to(torch.float64).cpu().numpy()
        dV, _, _ = ctx.solver.grad_density(G=G, rtol=ctx.rtol, maxit=ctx.maxit)
        return torch.from_numpy(dV).to(ctx.device), None, None, None, None, None


__all__ = ["EigenvalueSum", "Density", "hq"]
