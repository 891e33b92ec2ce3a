"""Mean Phi of a Monte Carlo study as a differentiable function of the
controller's tuning, for gradient-based tuning (the use the paper proposes
for its Monte Carlo study, Sec. VIII).

``pi_mean_phi(gains, study)``: mean_j Phi_j of a PI study at gains
(k_P, k_I, k_aw); the backward pass is the mean of the per-trajectory
discrete adjoints of the CUDA library (mc_pi_grad).

``nmpc_mean_phi(weights, study)``: mean_j Phi_j of an NMPC study at the
objective weights (Q_z, R_u, Q_n); the backward pass is the mean of the
per-trajectory tangents (mc_nmpc_grad: implicit differentiation of every
OCP's KKT point, exact derivatives of plant and CD-EKF).

Neither records a tape of torch ops.
"""
from __future__ import annotations

import torch

from . import mc


class PiMeanPhi(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gains: torch.Tensor, study: "mc.MonteCarlo", checkpoint_every: int = 20):
        kP, kI, kaw = (float(v) for v in gains.detach().cpu().tolist())
        study.set_pi_gains(kP, kI, kaw)
        study.pi_grad(checkpoint_every)
        st = study.stats()
        g = study.grad_mean()
        ctx.save_for_backward(torch.tensor(g, dtype=gains.dtype, device=gains.device))
        return torch.tensor(st["phi_mean"], dtype=gains.dtype, device=gains.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None


def pi_mean_phi(gains: torch.Tensor, study: "mc.MonteCarlo", checkpoint_every: int = 20):
    """Mean Phi of the PI study `study` at gains = (k_P, k_I, k_aw)."""
    return PiMeanPhi.apply(gains, study, checkpoint_every)


class NmpcMeanPhi(torch.autograd.Function):
    @staticmethod
    def forward(ctx, weights: torch.Tensor, study: "mc.MonteCarlo"):
        Qz, Ru, Qn = (float(v) for v in weights.detach().cpu().tolist())
        study.set_nmpc_weights(Qz, Ru, Qn)
        study.nmpc_grad()
        st = study.stats()
        g = study.grad_mean()
        ctx.save_for_backward(torch.tensor(g, dtype=weights.dtype, device=weights.device))
        return torch.tensor(st["phi_mean"], dtype=weights.dtype, device=weights.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None


def nmpc_mean_phi(weights: torch.Tensor, study: "mc.MonteCarlo"):
    """Mean Phi of the NMPC study `study` at weights = (Q_z, R_u, Q_n)."""
    return NmpcMeanPhi.apply(weights, study)
