"""torch.autograd access to the chirplet score and its adjoint kernel.

ChirpletScore(theta, residual, fs) returns s_b = <r_b, g(theta_b)> for the
unit-norm real chirplet of Eq. (1) at continuous parameters theta_b =
(tc [samples], fc [Hz], logDt, c [Hz/s]).  Forward and backward both come
from act_chirplet_score (one kernel computes the score, ds/dtheta and
g(theta) = ds/dr); backward only applies the chain rule to them.  This is
the differentiable handle Fig. 1's refinement step needs: maximising |s|
over theta with any torch optimiser refines a chirplet off the grid.
"""
from __future__ import annotations

import torch

from . import act


class ChirpletScore(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, residual: torch.Tensor, fs: float) -> torch.Tensor:
        if not (theta.is_cuda and residual.is_cuda):
            raise ValueError("ChirpletScore runs on the GPU: pass CUDA tensors")
        th = theta.detach().to(torch.float64).contiguous()
        r = residual.detach().to(torch.float32).contiguous()
        B, L = r.shape
        if th.shape != (B, 4):
            raise ValueError("theta must be [channels, 4]")
        score = torch.empty(B, dtype=torch.float64, device=r.device)
        grad = torch.empty((B, 4), dtype=torch.float64, device=r.device)
        atoms = torch.empty((B, L), dtype=torch.float32, device=r.device)
        act.act_chirplet_score(L, fs, th, r, B, score, grad, atoms)
        ctx.save_for_backward(grad, atoms)
        ctx.dtypes = (theta.dtype, residual.dtype)
        # the usual promotion of the inputs' dtypes (float64 with a float64 theta)
        return score.to(torch.promote_types(theta.dtype, residual.dtype))

    @staticmethod
    def backward(ctx, grad_score: torch.Tensor):
        grad, atoms = ctx.saved_tensors
        g_theta = (grad_score.to(torch.float64)[:, None] * grad).to(ctx.dtypes[0])
        g_res = (grad_score.to(torch.float32)[:, None] * atoms).to(ctx.dtypes[1])
        return g_theta, g_res, None


def chirplet_score(theta: torch.Tensor, residual: torch.Tensor, fs: float) -> torch.Tensor:
    """Differentiable s = <residual, g(theta)> per channel (see ChirpletScore)."""
    return ChirpletScore.apply(theta, residual, fs)
