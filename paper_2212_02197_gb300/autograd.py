"""Mean Phi of a Monte Carlo study as a differentiable function of the
controller's tuning, for gradient-based tuning (the use the paper proposes
for its Monte Carlo study, Sec. VIII).

``pi_mean_phi(gains, study)``: mean_j Phi_j of a PI study at gains
(k_P, k_I, k_aw); the backward pass is the mean of the per-trajectory
discrete adjoints of the CUDA library (mc_pi_grad).

``nmpc_mean_phi(weights, study)``: mean_j Phi_j of an NMPC study at the
objective weights (Q_z, R_u, Q_n); the backward pass is the mean of the
per-trajectory tangents (mc_nmpc_grad: implicit differentiation of every
OCP's KKT point, exact derivatives of plant and CD-EKF).  That tangent is the
derivative of the closed loop whose OCPs sit exactly at their KKT points.
The forward value is simulated with the OCPs stopped at the study's SQP
tolerance, and an SQP stopped early lags the exact solution map: at the
workload's 1e-5 the mean derivatives in Q_z and R_u differ from central
differences of the returned mean by about 15 %, at 1e-7 by a few per cent.
The function therefore warns when the study's tolerance is looser than 1e-7.

Neither records a tape of torch ops.
"""
from __future__ import annotations

import warnings

import torch

from . import mc

# SQP tolerance above which the NMPC forward value and its tangent part ways
_NMPC_GRAD_TOL = 1e-7


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
        tol = study.sqp_tol
        if tol is not None and tol > _NMPC_GRAD_TOL:
            warnings.warn(f"the study's OCPs stop at SQP tolerance {tol:g}; the gradient is "
                          f"that of OCPs at their exact KKT points, which the returned mean "
                          f"follows only to about the stopping error (use <= "
                          f"{_NMPC_GRAD_TOL:g} for a consistent pair)", stacklevel=3)
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
    """Mean Phi of the NMPC study `study` at weights = (Q_z, R_u, Q_n); its
    gradient is exact for OCPs solved to their KKT points (see the module
    notes: warns when the study's SQP tolerance is looser than 1e-7)."""
    return NmpcMeanPhi.apply(weights, study)
