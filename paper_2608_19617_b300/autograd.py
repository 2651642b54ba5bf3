"""Design field -> window objective as a torch.autograd.Function.

Forward runs consecutive windows (Alg. 1) until the window test of Eq. 26
holds or ``max_windows`` is reached and returns that window's J_eff (Eq. 27).
Backward runs the discrete adjoint over that window (Eqs. 35-39) and returns
dJ_eff/dgamma (Eq. 40, with gamma = 1 - phi) times the incoming gradient.
Both directions are the CUDA library's; torch only carries the tensors.
"""
from __future__ import annotations

import torch

from .binding import Solver


class WindowObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma: torch.Tensor, solver: Solver, max_windows: int = 0):
        g = gamma.detach().to(device=solver.device, dtype=torch.float32).contiguous()
        solver.set_design(g)
        rec = solver.run_until_converged(max_windows or None)
        ctx.solver = solver
        ctx.gdtype = gamma.dtype
        ctx.gdevice = gamma.device
        ctx.shape = gamma.shape
        return torch.tensor(rec[-1]["J"], dtype=torch.float64, device=gamma.device)

    @staticmethod
    def backward(ctx, grad_out):
        solver = ctx.solver
        solver.adjoint_window()
        g = torch.empty(solver.n, dtype=torch.float64, device=solver.device)
        solver.design_gradient(g)
        g = g.reshape(ctx.shape).to(device=ctx.gdevice)
        return (grad_out.to(torch.float64) * g).to(ctx.gdtype), None, None


def window_objective(gamma: torch.Tensor, solver: Solver, max_windows: int = 0) -> torch.Tensor:
    return WindowObjective.apply(gamma, solver, max_windows)
