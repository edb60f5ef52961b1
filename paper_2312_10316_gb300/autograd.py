"""torch.autograd.Function around the library's forward run and discrete adjoint.

``PhiOfD.apply(D, solver, ux, uy, phi0, steps, interval)`` runs `steps` TRT-R steps
(Eq. (14)) from g = g^eq(phi0, u) with the diffusivity field D (a CUDA float64 tensor
[ny][nx]) and returns phi at the last step; its backward returns dJ/dD through the
library's adjoint sweep (trtr_forward_record / trtr_adjoint, sqrt(steps) checkpoints).
All computation happens in the CUDA library; this module only passes tensors.
"""
from __future__ import annotations

import torch

from . import trtr as T


class PhiOfD(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D, solver: T.Solver, ux, uy, phi0, steps: int, interval: int = 0):
        solver.set_fields(ux, uy, D.detach().contiguous())
        solver.init_equilibrium(phi0)
        solver.forward_record(int(steps), int(interval))
        phi = torch.empty_like(D)
        solver.moments(phi)
        ctx.solver = solver
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        grad = torch.empty_like(grad_phi)
        ctx.solver.adjoint(grad_phi.detach().contiguous(), grad)
        return grad, None, None, None, None, None, None


def misfit_and_gradient(solver: T.Solver, ux, uy, D, phi0, phi_obs, steps: int, interval: int = 0):
    """J = 1/2 sum (phi - phi_obs)^2 after `steps` steps and dJ/dD (both on the device)."""
    Dv = D.detach().clone().requires_grad_(True)
    phi = PhiOfD.apply(Dv, solver, ux, uy, phi0, steps, interval)
    J = 0.5 * torch.sum((phi - phi_obs) ** 2)
    J.backward()
    return J.detach(), Dv.grad
