"""torch.autograd.Function over the unrolled A-MMMSE of amm_unrolled_*.

``unrolled_wsr(solver, H, gamma, alpha, sigma2, P, V0)`` returns WSR(V^T)
per instance (bits, float64) from T iterations with step sizes ``gamma``
(float32, T, shared by the batch) and the solver's fixed stage schedule;
its backward runs the CUDA adjoint and returns the gradients with respect
to ``H`` (complex64, real-gradient convention, which is torch's) and
``gamma``.  Argument marshalling only: both passes run in the library.
"""
from __future__ import annotations

import torch

from .amm import UnrolledSolver

__all__ = ["UnrolledSolver", "UnrolledAMMMSE", "unrolled_wsr"]


class UnrolledAMMMSE(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, gamma, alpha, sigma2, P, V0, solver: UnrolledSolver):
        H = H.contiguous()
        gamma = gamma.detach().to(torch.float32).contiguous()
        wsr = torch.empty(solver.batch, dtype=torch.float64, device=H.device)
        solver.forward(H.detach(), alpha.contiguous(), sigma2.contiguous(), P.contiguous(), V0.contiguous(), gamma,
                       wsr)
        ctx.solver = solver
        ctx.keep = (H, gamma)
        return wsr

    @staticmethod
    def backward(ctx, wsr_bar):
        solver = ctx.solver
        H, gamma = ctx.keep
        gamma_bar = torch.empty(solver.batch, solver.T, dtype=torch.float32, device=H.device)
        H_bar = torch.empty_like(H)
        solver.backward(wsr_bar.to(torch.float64).contiguous(), gamma_bar, H_bar)
        return H_bar, gamma_bar.sum(0), None, None, None, None, None


def unrolled_wsr(solver: UnrolledSolver, H, gamma, alpha, sigma2, P, V0):
    return UnrolledAMMMSE.apply(H, gamma, alpha, sigma2, P, V0, solver)
