"""Shared helpers of the parity tests: run the CUDA path and the oracle on the
same seeded inputs and compare."""
import numpy as np

from oracle import lbm as O


def f32_inputs(case):
    """Round the float inputs to FP32, the precision the C ABI takes them in,
    so that both sides see identical values."""
    return case.replace(gamma=case.gamma.astype(np.float32).astype(np.float64),
                        obj_weights=case.obj_weights.astype(np.float32).astype(np.float64),
                        inlet_u=case.inlet_u.astype(np.float32).astype(np.float64))


def rel_err(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def cosine(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def oracle_advance(pr, p, steps):
    g = pr.g()
    for _ in range(steps):
        _, _, p, _ = pr.step(p, g)
    return p


def fluid_moments(pr, p, case):
    rho, u = O.moments_of(pr.lat, pr.stream(p))
    fluid = case.gamma.reshape(-1) < 0.5
    return rho[fluid], u[:, fluid]


def initial_flow(pr, amp=0.04):
    """A smooth moving equilibrium (rho = 1): u_x = amp (1 + sin), u_y = amp/4 sin.
    Gives every case -- periodic ones included -- a nontrivial flow."""
    n = pr.n
    i = np.arange(n)
    x, y = i % pr.nx, (i // pr.nx) % pr.ny
    u = np.zeros((pr.lat.d, n))
    u[0] = amp * (1.0 + 0.5 * np.sin(2 * np.pi * y / pr.ny))
    u[1] = 0.25 * amp * np.sin(2 * np.pi * x / pr.nx)
    return O.equilibrium(pr.lat, np.ones(n), u)
