"""Pins of the MMA oracle (Svanberg 1987; the design update of Sec. 3.3).

* the convex approximation matches each function's value and gradient at the
  expansion point (central differences of the approximation, not its formula);
* the asymptote rules on numbers worked by hand;
* the subproblem's solution satisfies the KKT conditions of the primal
  subproblem, and equals an independent primal solve (SLSQP);
* whole MMA runs reach the closed-form optimum of min sum c_j / x_j subject to
  a volume bound, and keep a volume band feasible;
* planted mistakes (a dropped square in p, swapped asymptotes in the closed
  form) break these pins.
"""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import mma as M


def _random_problem(n=40, m=2, seed=3):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.2, 0.8, n)
    low, upp = x - rng.uniform(0.1, 0.5, n), x + rng.uniform(0.1, 0.5, n)
    fval = rng.standard_normal(m + 1)
    dfdx = rng.standard_normal((m + 1, n))
    return x, low, upp, fval, dfdx


def test_approximation_matches_value_and_gradient():
    x, low, upp, fval, dfdx = _random_problem()
    p, q, r = M.approximation(x, low, upp, fval, dfdx)
    assert np.allclose(M.approx_value(x, low, upp, p, q, r), fval, rtol=0, atol=1e-12)
    h = 1e-6
    for j in (0, 7, 23, 39):
        e = np.zeros_like(x)
        e[j] = h
        fd = (M.approx_value(x + e, low, upp, p, q, r) - M.approx_value(x - e, low, upp, p, q, r)) / (2 * h)
        assert np.allclose(fd, dfdx[:, j], rtol=1e-7, atol=1e-8), j
    # convex: second derivatives 2p/(U-x)^3 + 2q/(x-L)^3 >= 0 along every coordinate
    j, e = 5, np.zeros_like(x)
    e[5] = 1e-3
    second = (M.approx_value(x + e, low, upp, p, q, r) - 2 * fval + M.approx_value(x - e, low, upp, p, q, r))
    assert np.all(second >= -1e-12), j


def test_asymptote_rules_by_hand():
    xmin, xmax = np.zeros(3), np.ones(3)
    x = np.full(3, 0.5)
    # first two iterations: x -/+ 0.5 (xmax - xmin)
    lo, up = M.asymptotes(1, x, None, None, None, None, xmin, xmax)
    assert np.allclose(lo, 0.0) and np.allclose(up, 1.0)
    # k = 3: monotone (expand 1.2), oscillating (contract 0.7), stalled (keep)
    xold1 = np.array([0.4, 0.4, 0.5])
    xold2 = np.array([0.3, 0.45, 0.5])
    low = np.array([0.2, 0.2, 0.2])
    upp = np.array([0.7, 0.7, 0.8])
    lo, up = M.asymptotes(3, x, xold1, xold2, low, upp, xmin, xmax)
    assert np.allclose(lo, [0.5 - 1.2 * 0.2, 0.5 - 0.7 * 0.2, 0.5 - 1.0 * 0.3])
    assert np.allclose(up, [0.5 + 1.2 * 0.3, 0.5 + 0.7 * 0.3, 0.5 + 1.0 * 0.3])
    # distances kept within [0.01, 10] of the span
    lo, up = M.asymptotes(3, x, np.array([0.499995] * 3), np.array([0.49999] * 3), np.array([0.49999] * 3),
                          np.array([0.50001] * 3), xmin, xmax)
    assert np.allclose(lo, 0.49) and np.allclose(up, 0.51)
    alpha, beta = M.move_limits(x, np.full(3, 0.0), np.full(3, 1.0), np.full(3, 0.1), np.full(3, 0.9))
    assert np.allclose(alpha, 0.1) and np.allclose(beta, 0.9)
    alpha, beta = M.move_limits(x, np.full(3, 0.4), np.full(3, 0.6), xmin, xmax)
    assert np.allclose(alpha, 0.41) and np.allclose(beta, 0.59)


def _kkt_residual(z, y, lam, low, upp, alpha, beta, p, q, r, c=M.C_ART):
    """Largest violation of the KKT conditions of the subproblem."""
    f = M.approx_value(z, low, upp, p, q, r)
    P = p[0] + lam @ p[1:]
    Q = q[0] + lam @ q[1:]
    grad = P / (upp - z) ** 2 - Q / (z - low) ** 2          # d/dz of the Lagrangian
    scale = np.abs(grad).max() + 1e-300
    inside = (z > alpha + 1e-12) & (z < beta - 1e-12)
    at_lo, at_hi = z <= alpha + 1e-12, z >= beta - 1e-12
    res = [np.abs(grad[inside]).max(initial=0) / scale,
           max(0.0, -grad[at_lo].min(initial=0)) / scale,     # at alpha the Lagrangian may only rise
           max(0.0, grad[at_hi].max(initial=0)) / scale]
    g = f[1:] - y
    res.append(max(0.0, g.max()) / (1 + np.abs(f).max()))    # primal feasibility
    res.append(np.abs(lam * g).max() / (1 + np.abs(f).max()))   # complementary slackness
    res.append(np.abs(y - np.maximum(0, lam - c)).max())
    return max(res)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_subproblem_satisfies_kkt(seed):
    x, low, upp, fval, dfdx = _random_problem(seed=seed)
    xmin, xmax = np.zeros_like(x), np.ones_like(x)
    alpha, beta = M.move_limits(x, low, upp, xmin, xmax)
    # make both constraints bind: f_i(x) > 0 so that the unconstrained minimiser violates them
    fval[1:] = np.abs(fval[1:]) + 0.5
    p, q, r = M.approximation(x, low, upp, fval, dfdx)
    z, y, lam = M.solve_subproblem(x, low, upp, alpha, beta, p, q, r)
    assert np.all((z >= alpha) & (z <= beta))
    assert _kkt_residual(z, y, lam, low, upp, alpha, beta, p, q, r) < 1e-7


def test_subproblem_equals_a_primal_solve():
    """The dual method's z against SLSQP on the primal subproblem (one
    constraint, feasible without artificial variables)."""
    x, low, upp, fval, dfdx = _random_problem(n=20, m=1, seed=9)
    dfdx[1] = np.abs(dfdx[1]) + 0.1        # a volume-like constraint, increasing in every variable
    fval[1] = 0.05                          # slightly violated at x: it binds
    xmin, xmax = np.zeros_like(x), np.ones_like(x)
    alpha, beta = M.move_limits(x, low, upp, xmin, xmax)
    p, q, r = M.approximation(x, low, upp, fval, dfdx)
    z, y, lam = M.solve_subproblem(x, low, upp, alpha, beta, p, q, r)
    assert y[0] == 0 and lam[0] > 0
    cons = {"type": "ineq", "fun": lambda v: -M.approx_value(v, low, upp, p, q, r)[1]}
    res = minimize(lambda v: M.approx_value(v, low, upp, p, q, r)[0], x, method="SLSQP",
                   bounds=list(zip(alpha, beta)), constraints=[cons], options={"ftol": 1e-12, "maxiter": 500})
    assert res.status in (0, 8)             # 8: stopped at the precision limit of its line search
    assert np.abs(z - res.x).max() < 1e-5


def test_mma_reaches_the_closed_form_optimum():
    """min sum c_j / x_j subject to mean(x) <= V on [1e-3, 1]: x_j ~ sqrt(c_j)."""
    rng = np.random.default_rng(4)
    n, V = 30, 0.3
    c = rng.uniform(1.0, 4.0, n)
    want = V * n * np.sqrt(c) / np.sqrt(c).sum()
    opt = M.MMA(np.full(n, 1e-3), np.ones(n))
    x = np.full(n, 0.5)
    for _ in range(40):
        f = np.array([(c / x).sum(), x.mean() - V])
        df = np.vstack([-c / x ** 2, np.full(n, 1.0 / n)])
        x, lam = opt.update(x, f, df)
    assert np.abs(x - want).max() < 1e-6
    assert abs(x.mean() - V) < 1e-8


def test_mma_keeps_a_volume_band():
    """A band Vmin <= mean(x) <= Vmax as two constraints (the paper's volume
    bounds): minimising sum_j x_j^2 w_j pushes the volume down to Vmin."""
    rng = np.random.default_rng(8)
    n, vmin, vmax = 25, 0.4, 0.45
    w = rng.uniform(0.5, 2.0, n)
    opt = M.MMA(np.zeros(n), np.ones(n))
    x = rng.uniform(0.6, 0.9, n)
    for _ in range(60):
        v = x.mean()
        f = np.array([(w * x * x).sum(), v - vmax, vmin - v])
        df = np.vstack([2 * w * x, np.full(n, 1.0 / n), np.full(n, -1.0 / n)])
        x, lam = opt.update(x, f, df)
    assert abs(x.mean() - vmin) < 1e-7
    want = vmin * n * (1 / w) / (1 / w).sum()      # x_j ~ 1/w_j at the lower bound
    assert np.abs(x - want).max() < 1e-6


def test_dropped_square_in_p_is_caught(monkeypatch):
    x, low, upp, fval, dfdx = _random_problem()

    def mutant(x, low, upp, fval, dfdx):
        ux, xl = upp - x, x - low
        p = ux * np.maximum(dfdx, 0.0)
        q = xl ** 2 * np.maximum(-dfdx, 0.0)
        return p, q, fval - (p / ux + q / xl).sum(axis=1)

    monkeypatch.setattr(M, "approximation", mutant)
    p, q, r = M.approximation(x, low, upp, fval, dfdx)
    e = np.zeros_like(x)
    e[3] = 1e-6
    fd = (M.approx_value(x + e, low, upp, p, q, r) - M.approx_value(x - e, low, upp, p, q, r)) / 2e-6
    assert not np.allclose(fd, dfdx[:, 3], rtol=1e-7, atol=1e-8)


def test_swapped_asymptotes_in_the_closed_form_are_caught(monkeypatch):
    x, low, upp, fval, dfdx = _random_problem(seed=2)
    fval[1:] = np.abs(fval[1:]) + 0.5
    xmin, xmax = np.zeros_like(x), np.ones_like(x)
    alpha, beta = M.move_limits(x, low, upp, xmin, xmax)
    p, q, r = M.approximation(x, low, upp, fval, dfdx)
    orig = M.primal_of_dual

    def mutant(lam, x, low, upp, alpha, beta, p, q):
        return orig(lam, x, upp, low, alpha, beta, p, q)

    monkeypatch.setattr(M, "primal_of_dual", mutant)
    z, y, lam = M.solve_subproblem(x, low, upp, alpha, beta, p, q, r)
    assert _kkt_residual(z, y, lam, low, upp, alpha, beta, p, q, r) > 1e-3
