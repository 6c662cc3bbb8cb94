"""torch.autograd.Function over the unrolled A-MMMSE of amm_unrolled_*.

``unrolled_wsr(solver, H, gamma, alpha, sigma2, P, V0)`` returns WSR(V^T)
per instance (bits, float64) from T iterations with step sizes ``gamma``
(float32, T, shared by the batch) and the solver's fixed stage schedule;
its backward runs the CUDA adjoint and returns the gradients with respect
to ``H`` (complex64, real-gradient convention, which is torch's) and
``gamma``.  Argument marshalling only: both passes run in the library.
The adjoint reads the checkpoints of the solver's last forward; a graph
whose forward is no longer the last one on its solver recomputes it before
its backward, so several graphs may share one solver.
"""
from __future__ import annotations

import torch

from .amm import UnrolledSolver

__all__ = ["UnrolledSolver", "UnrolledAMMMSE", "unrolled_wsr"]


class UnrolledAMMMSE(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, gamma, alpha, sigma2, P, V0, solver: UnrolledSolver):
        Hc = H.detach().contiguous()
        g32 = gamma.detach().to(torch.float32).contiguous()
        args = (Hc, alpha.contiguous(), sigma2.contiguous(), P.contiguous(), V0.contiguous(), g32)
        wsr = torch.empty(solver.batch, dtype=torch.float64, device=H.device)
        solver.forward(*args, wsr)
        ctx.solver = solver
        ctx.generation = solver.generation
        # the inputs themselves are saved, so torch's version check catches an
        # in-place edit between forward and backward; the contiguous copies
        # (the same tensors when no copy was needed) are what the kernels read
        ctx.save_for_backward(H, gamma, *args)
        return wsr

    @staticmethod
    def backward(ctx, wsr_bar):
        solver = ctx.solver
        saved = ctx.saved_tensors
        args = saved[2:]
        if solver.generation != ctx.generation:
            # another forward ran on this solver since (a second loss, a
            # validation pass): its checkpoints are that call's, so this
            # graph's forward is recomputed first (same inputs, same result)
            solver.forward(*args, torch.empty(solver.batch, dtype=torch.float64, device=args[0].device))
        Hc = args[0]
        gamma_bar = torch.empty(solver.batch, solver.T, dtype=torch.float32, device=Hc.device)
        H_bar = torch.empty_like(Hc)
        solver.backward(wsr_bar.to(torch.float64).contiguous(), gamma_bar, H_bar)
        return H_bar, gamma_bar.sum(0), None, None, None, None, None


def unrolled_wsr(solver: UnrolledSolver, H, gamma, alpha, sigma2, P, V0):
    return UnrolledAMMMSE.apply(H, gamma, alpha, sigma2, P, V0, solver)
