"""Differentiable NMPC solve: torch.autograd.Function around nmpc_solve and
nmpc_sensitivity.

forward(x0, setpoint, u_prev) sets the parameters of one instance, solves, and
returns the primal solution y* (device tensor).  backward(dl/dy*) calls the
library's adjoint, which reuses the stored Cholesky factor with iterative
refinement, and returns dl/dx0 and dl/dsetpoint (no gradient for u_prev).
The backward pass must run before the solver is used again: it differentiates
the solver's current converged point.
"""
from __future__ import annotations

import torch


class NmpcSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, instance, x0, setpoint, u_prev, warm=False):
        solver.set_params(instance=instance, x0=x0.detach().contiguous(), setpoint=setpoint.detach().contiguous(),
                          u_prev=u_prev.detach().contiguous())
        info = solver.solve(warm=warm)[instance]
        if info["status"] != 0:
            raise RuntimeError(f"NMPC solve failed: {info}")
        n, _, _ = solver.dims[instance]
        y = torch.empty(n, dtype=torch.float64, device=x0.device)
        solver.get_solution(instance, out=(y, None))
        ctx.solver, ctx.instance = solver, instance
        ctx.x0_shape, ctx.sp_shape = x0.shape, setpoint.shape
        return y

    @staticmethod
    def backward(ctx, grad_y):
        dx0 = torch.empty(ctx.x0_shape, dtype=torch.float64, device=grad_y.device)
        dsp = torch.empty(ctx.sp_shape, dtype=torch.float64, device=grad_y.device)
        ctx.solver.sensitivity(ctx.instance, grad_y.contiguous(), dx0, dsp)
        return None, None, dx0, dsp, None, None


def nmpc_solve(solver, x0, setpoint, u_prev, instance=0, warm=False):
    """y* = argmin of the instance's OCP, differentiable in x0 and setpoint."""
    return NmpcSolve.apply(solver, instance, x0, setpoint, u_prev, warm)
