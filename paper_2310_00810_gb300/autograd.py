"""torch.autograd integration: the final-step loss of an LBM solve as a
differentiable function of the inlet density and tau.

Forward runs ``lbm_forward`` (T steps from rest, writing the sqrt(T)
checkpoints into the solver's workspace) and ``lbm_loss_grad`` (loss and its
seed lambda^T).  Backward runs ``lbm_adjoint``: the hand-written reverse sweep
that recomputes each checkpoint segment and steps the adjoint backwards
(it stands in for the Taichi tape of the paper, section 2.2).  Both are the
library's CUDA kernels; this module only wires them into autograd.

The workspace holds the checkpoints of the last forward: call ``backward``
before running another forward on the same solver.
"""
from __future__ import annotations

import torch

from . import lbm


class LBMLoss(torch.autograd.Function):
    """loss = LBMLoss.apply(rho_in, tau, solver, rho_out, u_target, roi)

    rho_in: float64 [n_in] (1 for a constant head, ny*nz for a profile);
    tau: float64 [1]; u_target: float64 [D, ...]; roi: uint8 [...] or None.
    Returns a float64 [1] tensor; gradients flow to rho_in and tau."""

    @staticmethod
    def forward(ctx, rho_in, tau, solver, rho_out, u_target, roi):
        rho_in = rho_in.detach().contiguous()
        tau = tau.detach().contiguous()
        f = solver.forward(rho_in, tau, rho_out)
        loss, lam = solver.loss_grad(f, u_target, roi)
        ctx.solver = solver
        ctx.rho_out = float(rho_out)
        ctx.save_for_backward(rho_in, tau, lam)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        rho_in, tau, lam = ctx.saved_tensors
        g_in, g_tau = ctx.solver.adjoint(rho_in, tau, ctx.rho_out, lam)
        scale = grad_loss.reshape(())
        return g_in * scale, g_tau * scale, None, None, None, None


def lbm_loss(rho_in, tau, solver: lbm.Solver, rho_out: float, u_target, roi=None):
    """Functional form of LBMLoss."""
    return LBMLoss.apply(rho_in, tau, solver, rho_out, u_target, roi)
