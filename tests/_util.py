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


def decaying_stream_window(q, window_len, sample_every, sample_from, g0=0.3, u0=0.03,
                           monitor_u=0.05, monitor_l=7.0, rho_out=1.0):
    """One oracle window on a uniform stream through a uniform partial solid in a
    periodic box, next to its closed form.

    Streaming leaves a uniform field unchanged, the collision keeps rho and m,
    and the blend of Eq. 23 scales m by (1 - 2g) exactly, so the field pulled
    at step k of the window has rho = 1 and u = (1 - 2g)^k u0 e_x.  Then
      velocity-deviation sample (u_ref = 0, weights 1/N):  ((1 - 2g)^k u0)^2,
      drag monitor (Eq. 25 over Eq. 44's F_x, summed over the N nodes):
          -2 g (1 - 2g)^k u0 N / (1/2 rho_0 U^2 L),
    and the window means of Eq. 42 weight the samples k = s0, s0 + dW, ... by
    dW / (|W| - s0).  Returns (J, M) of the oracle and of the closed form."""
    from paper_2608_19617_b300 import inputs as I
    nx, ny, nz = 7, 5, (4 if q == 19 else 1)
    case = I.periodic_box(nx, ny, nz, lattice=q, gamma=np.full((nz, ny, nx), g0))
    case = case.replace(obj_kind=I.OBJ_VELOCITY_DEV, obj_uref=(0.0, 0.0, 0.0), monitor_kind=I.MON_DRAG,
                        monitor_u=monitor_u, monitor_l=monitor_l, rho_out=rho_out, window_len=window_len,
                        sample_every=sample_every, sample_from=sample_from)
    pr = O.Problem(case)
    u = np.zeros((pr.lat.d, pr.n))
    u[0] = u0
    p0 = O.equilibrium(pr.lat, np.ones(pr.n), u)
    _, J, M, _ = pr.run_window(p0, store=False)
    g = float(pr.g()[0])
    ks = np.arange(sample_from, window_len, sample_every)
    decay = (1.0 - 2.0 * g) ** ks
    J_want = float(np.mean((decay * u0) ** 2))
    M_want = float(np.mean(-2.0 * g * decay * u0 * pr.n / (0.5 * rho_out * monitor_u ** 2 * monitor_l)))
    return J, M, J_want, M_want
