"""Plain FP64 CPU oracle of the Method of Moving Asymptotes (Svanberg 1987).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only the
tests use it.  It shares no code with the CUDA path.

The paper updates its design variables with MMA under the volume constraint
(Sec. 3.3, topology optimization procedure, citing Svanberg 1987).  One MMA
iteration, as written out here from that method:

1. moving asymptotes L_j < x_j < U_j: at the first two iterations
   x_j -/+ s0 (xmax_j - xmin_j); afterwards they contract by s_slow where the
   last two changes of x_j have opposite signs (oscillation), expand by s_fast
   where they have the same sign, and keep their distance otherwise, each kept
   within [0.01, 10] (xmax_j - xmin_j) of x_j;
2. move limits alpha_j = max(xmin_j, L_j + a (x_j - L_j)),
   beta_j = min(xmax_j, U_j - a (U_j - x_j)), a = 0.1;
3. convex separable approximations of the objective (i = 0) and of the
   constraints f_i <= 0 (i = 1..m) at x:
   f~_i(z) = r_i + sum_j p_ij / (U_j - z_j) + q_ij / (z_j - L_j),
   p_ij = (U_j - x_j)^2 max(0, df_i/dx_j), q_ij = (x_j - L_j)^2 max(0, -df_i/dx_j),
   r_i = f_i(x) - sum_j p_ij / (U_j - x_j) + q_ij / (x_j - L_j),
   which match f_i and its gradient at z = x;
4. the subproblem min f~_0(z) + sum_i (c_i y_i + y_i^2 / 2) subject to
   f~_i(z) - y_i <= 0, y_i >= 0, alpha <= z <= beta, solved by its dual
   (Svanberg's dual method): for multipliers lam >= 0 each z_j minimises
   P_j / (U_j - z_j) + Q_j / (z_j - L_j) with P_j = p_0j + lam.p_j,
   Q_j = q_0j + lam.q_j, in closed form
   z_j = (sqrt(P_j) L_j + sqrt(Q_j) U_j) / (sqrt(P_j) + sqrt(Q_j)) clipped to
   [alpha_j, beta_j]; y_i = max(0, lam_i - c_i); the concave dual W(lam) is
   maximised over lam >= 0 (here by a bounded quasi-Newton library routine).

The artificial variables y_i (cost c_i = 1000) keep every subproblem feasible;
they are the standard safeguard of the method and zero whenever the
approximated constraints can be met.  Readings where Svanberg 1987 leaves a
choice (s0 = 0.5, s_slow = 0.7, s_fast = 1.2, a = 0.1, the [0.01, 10] bounds
of the asymptote distance, c_i) are listed in the design notes.

Pins (tests/test_oracle_mma.py): first-order agreement of the approximation
with finite differences, the asymptote rules on hand-worked numbers, the
subproblem's KKT conditions and an SLSQP solve of its primal, the closed-form
optimum of min sum c/x under a volume bound, and planted mistakes that must
fail them.
"""

from __future__ import annotations

import numpy as np
from scipy.optimize import minimize

S_INIT, S_SLOW, S_FAST, ALBEFA, C_ART = 0.5, 0.7, 1.2, 0.1, 1000.0


def asymptotes(k, x, xold1, xold2, low, upp, xmin, xmax):
    """Step 1: asymptotes of iteration k (k = 1, 2, ...)."""
    span = xmax - xmin
    if k <= 2:
        return x - S_INIT * span, x + S_INIT * span
    sign = (x - xold1) * (xold1 - xold2)
    fac = np.where(sign < 0, S_SLOW, np.where(sign > 0, S_FAST, 1.0))
    lo = x - fac * (xold1 - low)
    up = x + fac * (upp - xold1)
    lo = np.clip(lo, x - 10.0 * span, x - 0.01 * span)
    up = np.clip(up, x + 0.01 * span, x + 10.0 * span)
    return lo, up


def move_limits(x, low, upp, xmin, xmax):
    """Step 2."""
    return np.maximum(xmin, low + ALBEFA * (x - low)), np.minimum(xmax, upp - ALBEFA * (upp - x))


def approximation(x, low, upp, fval, dfdx):
    """Step 3: p, q [m+1][n] and r [m+1] for fval [m+1] and dfdx [m+1][n]."""
    ux, xl = upp - x, x - low
    p = ux ** 2 * np.maximum(dfdx, 0.0)
    q = xl ** 2 * np.maximum(-dfdx, 0.0)
    r = fval - (p / ux + q / xl).sum(axis=1)
    return p, q, r


def approx_value(z, low, upp, p, q, r):
    """f~_i(z) for every i."""
    return r + (p / (upp - z) + q / (z - low)).sum(axis=1)


def primal_of_dual(lam, x, low, upp, alpha, beta, p, q):
    """z(lam): the closed-form minimiser of each separable term, clipped.  A
    variable that no term depends on (P = Q = 0) stays at x."""
    P = p[0] + lam @ p[1:]
    Q = q[0] + lam @ q[1:]
    sp, sq = np.sqrt(P), np.sqrt(Q)
    with np.errstate(invalid="ignore", divide="ignore"):
        z = np.where(sp + sq > 0, (sp * low + sq * upp) / (sp + sq), x)
    return np.clip(z, alpha, beta)


def dual_value(lam, x, low, upp, alpha, beta, p, q, r, c=C_ART):
    """W(lam) and its gradient (concave; Danskin: the gradient is the
    constraint values at z(lam), y(lam))."""
    z = primal_of_dual(lam, x, low, upp, alpha, beta, p, q)
    f = approx_value(z, low, upp, p, q, r)
    y = np.maximum(0.0, lam - c)
    W = f[0] + lam @ (f[1:] - y) + c * y.sum() + 0.5 * (y * y).sum()
    return W, f[1:] - y, z, y


def solve_subproblem(x, low, upp, alpha, beta, p, q, r, c=C_ART):
    """Step 4: maximise the dual; return z, y and lam."""
    m = len(r) - 1

    def neg(lam):
        W, g, _, _ = dual_value(lam, x, low, upp, alpha, beta, p, q, r, c)
        return -W, -g

    res = minimize(neg, np.zeros(m), jac=True, method="L-BFGS-B", bounds=[(0.0, None)] * m,
                   options={"ftol": 1e-16, "gtol": 1e-13, "maxiter": 10000, "maxcor": 30})
    lam = np.maximum(res.x, 0.0)
    _, _, z, y = dual_value(lam, x, low, upp, alpha, beta, p, q, r, c)
    return z, y, lam


class MMA:
    """State of an MMA run: the last two iterates and asymptotes."""

    def __init__(self, xmin, xmax):
        self.xmin = np.asarray(xmin, np.float64)
        self.xmax = np.asarray(xmax, np.float64)
        self.k = 0
        self.xold1 = self.xold2 = self.low = self.upp = None

    def update(self, x, fval, dfdx):
        """One iteration from the point x with f_i(x) = fval[i] (i = 0 the
        objective, 1..m constraints f_i <= 0) and gradients dfdx [m+1][n].
        Returns the next point and the subproblem's multipliers."""
        x = np.asarray(x, np.float64)
        self.k += 1
        low, upp = asymptotes(self.k, x, self.xold1, self.xold2, self.low, self.upp, self.xmin, self.xmax)
        alpha, beta = move_limits(x, low, upp, self.xmin, self.xmax)
        p, q, r = approximation(x, low, upp, np.asarray(fval, np.float64), np.asarray(dfdx, np.float64))
        z, y, lam = solve_subproblem(x, low, upp, alpha, beta, p, q, r)
        self.xold2, self.xold1 = self.xold1, x.copy()
        self.low, self.upp = low, upp
        self.last = dict(low=low, upp=upp, alpha=alpha, beta=beta, p=p, q=q, r=r, y=y, lam=lam)
        return z, lam
