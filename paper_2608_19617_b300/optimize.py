"""The topology optimization loop (Alg. 2; Sec. 3.3, topology optimization procedure).

Each iteration, for the raw design variables x in [0, 1]:

1. the physical design gamma from x through the density filter (radius r)
   and the Heaviside projection (threshold eta, steepness beta: 2 at the
   start, doubled every 10 iterations up to 16) -- lbm_set_design_filtered;
2. windows of the flow until the consecutive-window test of Eq. 26 holds
   (Alg. 1), continuing from the previous design's flow;
3. the adjoint over that representative window and dJ_eff/dx through the
   chain rule of the filter and projection;
4. the volume V = mean gamma over the design box (the paper's
   (1/n_D) sum (1 - phi)) and its gradient, through the same chain rule;
5. an MMA update of x (Svanberg 1987) under Vmin <= V <= Vmax, posed as the
   two constraints V/Vmax - 1 <= 0 and 1 - V/Vmin <= 0, with the objective
   scaled by |J_eff| of the first iteration.

The loop stops after n_max iterations or when the relative change of J_eff
falls below eps_o.  Every step runs in the library (liblbmadj.so): this
module only sequences the calls.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def design_mask(case) -> np.ndarray:
    """1 inside the design box, 0 outside, as a flat [N] array."""
    m = np.zeros((case.nz, case.ny, case.nx))
    x0, x1, y0, y1, z0, z1 = case.design_box
    m[z0:z1, y0:y1, x0:x1] = 1.0
    return m.reshape(-1)


def optimize(case, *, n_max=60, eps_o=5e-3, vmin=0.014, vmax=0.016, radius=4.0, eta=0.5, beta0=2.0,
             beta_max=16.0, beta_every=10, precision=B.LBM_FP32, max_windows=None, x0=None, log=None):
    """Run the loop on ``case``; returns (history, final raw design x as numpy)."""
    import torch

    sol = B.Solver(case, precision)
    n = case.n
    mask = design_mask(case)
    n_d = float(mask.sum())
    x = torch.tensor(np.asarray(case.gamma if x0 is None else x0, np.float64).reshape(-1), device=sol.device)
    # variables outside the design box carry no sensitivity and stay where they are
    opt = B.Mma(np.zeros(n), np.ones(n), 2, device=sol.device, stream=sol.stream)
    history, j_scale, j_prev = [], None, None
    try:
        for it in range(n_max):
            beta = min(beta_max, beta0 * 2.0 ** (it // beta_every))
            sol.set_design_filtered(x.float().contiguous(), radius, beta, eta)
            rec = sol.run_until_converged(max_windows)
            j_eff = sol.adjoint_window()
            dj = sol.design_gradient_filtered()
            vol = sol.design_volume()
            dv = sol.filter_chain_rule(mask / n_d)
            if j_scale is None:
                j_scale = abs(j_eff) if j_eff != 0 else 1.0
            fval = np.array([j_eff / j_scale, vol / vmax - 1.0, 1.0 - vol / vmin])
            dfdx = np.stack([dj / j_scale, dv / vmax, -dv / vmin])
            lam = opt.update(x, fval, dfdx)
            row = dict(iteration=it, beta=beta, J=j_eff, volume=vol, windows=len(rec),
                       converged=bool(rec[-1]["converged"]), ratio=float(rec[-1]["ratio"]), lam=lam.tolist())
            history.append(row)
            if log:
                log(row)
            if j_prev is not None and abs(j_eff - j_prev) <= eps_o * abs(j_eff):
                break
            j_prev = j_eff
        return history, x.cpu().numpy()
    finally:
        opt.close()
        sol.close()
