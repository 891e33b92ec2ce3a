"""Mean Phi of a PI Monte Carlo study as a differentiable function of the
gains, for tuning by gradient methods (the use the paper proposes for its
Monte Carlo study, Sec. VIII).

``pi_mean_phi(gains, study)`` returns mean_j Phi_j over the study's finite
trajectories; its backward pass is the mean of the per-trajectory discrete
adjoints computed by the CUDA library (mc_pi_grad), not a tape of torch ops.
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
