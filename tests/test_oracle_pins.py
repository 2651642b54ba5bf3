"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
conservation laws, invariants, values the paper prints, or complex-step
derivatives of its own forward map (exact to rounding).  No GPU is used.
"""
import json
import os

import numpy as np
import pytest

from oracle import lbm as O
from paper_2608_19617_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


def _random_state(lat, n, amp=0.02, u_amp=0.05, rng=RNG):
    """Equilibrium at random (rho, u) plus a random non-equilibrium part."""
    rho = 1.0 + 0.05 * rng.standard_normal(n)
    u = u_amp * rng.standard_normal((lat.d, n))
    return O.equilibrium(lat, rho, u) + amp * lat.w[:, None] * rng.standard_normal((lat.q, n))


# ---------------------------------------------------------------- lattice --

@pytest.mark.parametrize("q", [9, 19])
def test_lattice_isotropy(q):
    """Moment identities of the weights up to fourth order (textbook closed form)."""
    lat = O.Lattice(q)
    c, w, d = lat.c, lat.w, lat.d
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ c).max() < 1e-15
    np.testing.assert_allclose(np.einsum("a,ap,aq->pq", w, c, c), O.CS2 * np.eye(d), atol=1e-15)
    m4 = np.einsum("a,ap,aq,ar,as->pqrs", w, c, c, c, c)
    e = np.eye(d)
    iso = O.CS4 * (np.einsum("pq,rs->pqrs", e, e) + np.einsum("pr,qs->pqrs", e, e)
                   + np.einsum("ps,qr->pqrs", e, e))
    np.testing.assert_allclose(m4, iso, atol=1e-15)
    for a in range(q):
        assert (lat.c3[lat.opp[a]] == -lat.c3[a]).all()


def test_d2q9_order_is_the_papers():
    """Velocity order of Sec. 2.1.1, Eq. 2."""
    lat = O.Lattice(9)
    expect = np.array([[0, 1, 0, -1, 0, 1, -1, -1, 1], [0, 0, 1, 0, -1, 1, 1, -1, -1]]).T
    assert (lat.c3[:, :2] == expect).all()
    np.testing.assert_allclose(lat.w, [4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36])


@pytest.mark.parametrize("q", [9, 19])
def test_equilibrium_moments(q):
    """Eq. 3 reproduces rho, rho u and rho cs^2 I + rho u u exactly."""
    lat = O.Lattice(q)
    n = 50
    rho = 1 + 0.1 * RNG.standard_normal(n)
    u = 0.1 * RNG.standard_normal((lat.d, n))
    feq = O.equilibrium(lat, rho, u)
    np.testing.assert_allclose(feq.sum(0), rho, rtol=1e-14)
    np.testing.assert_allclose(lat.c.T @ feq, rho * u, atol=1e-15)
    m2 = np.einsum("ap,aq,an->pqn", lat.c, lat.c, feq)
    expect = O.CS2 * rho * np.eye(lat.d)[..., None] + rho * np.einsum("pn,qn->pqn", u, u)
    np.testing.assert_allclose(m2, expect, atol=1e-14)


# -------------------------------------------------------------- collision --

@pytest.mark.parametrize("q", [9, 19])
def test_collision_invariants(q):
    """Collision conserves mass and momentum; the regularized part is the Hermite
    projection: its second moment is (1 - 1/tau_eff) Pi (Eq. 16)."""
    lat = O.Lattice(q)
    f = _random_state(lat, 64)
    h, aux = O.collide(lat, f, 0.52, 0.15)
    np.testing.assert_allclose(h.sum(0), f.sum(0), rtol=1e-14)
    np.testing.assert_allclose(lat.c.T @ h, lat.c.T @ f, atol=1e-15)
    m2neq = np.einsum("ap,aq,an->pqn", lat.c, lat.c, h - aux["feq"])
    np.testing.assert_allclose(m2neq, (1 - 1 / aux["tau_eff"]) * aux["pi"], atol=1e-15)
    # the regularized part also has no ghost (third-order diagonal) content left
    # beyond what the Hermite basis carries: its zeroth and first moments vanish
    hn = h - aux["feq"]
    assert np.abs(hn.sum(0)).max() < 1e-15 and np.abs(lat.c.T @ hn).max() < 1e-15


@pytest.mark.parametrize("q", [9, 19])
def test_tau_eff_solves_the_les_closure(q):
    """Eq. 14 is the closed-form solution of Eqs. 9-12: check the implicit
    definition tau_eff = (nu + (Cs)^2 |S|)/cs^2 + 1/2 with S from Eq. 12."""
    lat = O.Lattice(q)
    f = _random_state(lat, 64, amp=0.05)
    tau, cs = 0.51, 0.17
    h, aux = O.collide(lat, f, tau, cs)
    te, rho, pi = aux["tau_eff"], aux["rho"], aux["pi"]
    S = -pi / (2 * rho * O.CS2 * te)                        # Eq. 12
    snorm = np.sqrt(2 * (S * S).sum(axis=(0, 1)))          # |S| below Eq. 9
    nu = (tau - 0.5) * O.CS2                                # Eq. 8
    te_implicit = (nu + cs ** 2 * snorm) / O.CS2 + 0.5      # Eqs. 9-11
    np.testing.assert_allclose(te, te_implicit, rtol=1e-14)
    assert (te > tau).all()


def test_tau_eff_without_model_is_tau():
    lat = O.Lattice(9)
    f = _random_state(lat, 10)
    _, aux = O.collide(lat, f, 0.7, 0.0)
    np.testing.assert_allclose(aux["tau_eff"], 0.7, rtol=0, atol=0)


def test_g_interpolation():
    """g(phi) of Sec. 2.2: g(1)=0 (fluid), g(0)=1/2 (solid), decreasing, convex."""
    phi = np.linspace(0, 1, 101)
    g = O.g_of_phi(phi, 0.1, 0.5)
    assert g[0] == 0.5 and abs(g[-1]) < 1e-16
    assert (np.diff(g) < 0).all() and (np.diff(g, 2) > 0).all()
    h = 1e-30
    dg_cs = (O.g_of_phi(phi + 1j * h, 0.1, 0.5)).imag / h
    np.testing.assert_allclose(O.dg_dphi(phi, 0.1, 0.5), dg_cs, rtol=1e-14)


@pytest.mark.parametrize("q", [9, 19])
def test_partial_bounce_back_limits(q):
    """At a solid node (phi=0) with the paper's g=1/2 the blended field is
    symmetric (zero momentum); with g_max=1 it is the exact swap h_abar."""
    lat = O.Lattice(q)
    h = _random_state(lat, 8)
    g_half = O.g_of_phi(np.zeros(8), 0.1, 0.5)
    p = O.blend(lat, h, g_half)
    np.testing.assert_allclose(p, p[lat.opp], atol=0)
    assert np.abs(lat.c.T @ p).max() < 1e-16
    np.testing.assert_allclose(p.sum(0), h.sum(0), rtol=1e-15)
    g_one = O.g_of_phi(np.zeros(8), 0.1, 1.0)
    assert (O.blend(lat, h, g_one) == h[lat.opp]).all()
    # at a fluid node nothing happens
    g_fluid = O.g_of_phi(np.ones(8), 0.1, 0.5)
    np.testing.assert_allclose(O.blend(lat, h, g_fluid), h, atol=1e-17)


# --------------------------------------------------------------- boundary --

def test_zouhe_and_wall_rules_fix_their_moments():
    """After streaming + Eqs. 19-21: inlet nodes carry u=(u0,0), outlet nodes
    rho = rho0 and u_y = 0, top/bottom wall nodes u_y = 0."""
    case = I.small_channel(12, 7, profile="parabolic", u_in=0.06, outlet=I.OUTLET_P)
    case = case.replace(rho_out=1.02)
    pr = O.Problem(case)
    p = _random_state(pr.lat, pr.n)
    f = pr.stream(p)
    rho, u = O.moments_of(pr.lat, f)
    cls = case.node_class.reshape(-1)
    x = np.arange(pr.n) % pr.nx
    y = np.arange(pr.n) // pr.nx
    inl = cls == I.INLET
    np.testing.assert_allclose(u[0, inl], case.inlet_u.reshape(-1)[y[inl]], atol=1e-15)
    np.testing.assert_allclose(u[1, inl], 0, atol=1e-15)
    out = cls == I.OUTLET_P
    np.testing.assert_allclose(rho[out], 1.02, atol=1e-15)
    np.testing.assert_allclose(u[1, out], 0, atol=1e-15)
    wall = (cls == I.WALL) & (x > 0) & (x < pr.nx - 1)
    np.testing.assert_allclose(u[1, wall], 0, atol=1e-16)


def _local_block(pr, node, unknowns):
    """Coefficients B[u][k] of f_u(node) in terms of the known f_k(node)."""
    n, S = pr.n, pr.S.tocsr()
    x, y, z = node % pr.nx, (node // pr.nx) % pr.ny, node // (pr.nx * pr.ny)
    B = {}
    for u in unknowns:
        row = S.getrow(u * n + node)
        for k in range(pr.lat.q):
            if k in unknowns:
                continue
            src = pr._source(np.array([x]), np.array([y]), np.array([z]), k)[0]
            B[(u, k)] = row[0, k * n + src]
    return B


def test_adjoint_boundary_rules_match_the_paper():
    """The transposes of the oracle's forward inlet/outlet/wall rules carry the
    coefficients the paper prints for the adjoint rules (Eqs. 37-39)."""
    gold = json.load(open(os.path.join(GOLDEN, "adjoint_zouhe_bc.json")))
    case = I.small_channel(8, 6, u_in=0.07, outlet=I.OUTLET_P)
    pr = O.Problem(case)
    u0 = 0.07
    chi = u0 / (1 - u0)
    y = 2
    for side, node, unk, zero in (("inlet", y * pr.nx, (1, 5, 8), "inlet_zero"),
                                  ("outlet", y * pr.nx + pr.nx - 1, (3, 6, 7), "outlet_zero")):
        assert tuple(gold[zero]) == unk
        B = _local_block(pr, node, unk)
        # transpose: lambda_hat_k = lambda_k + sum_u B[u][k] lambda_u
        got = {}
        for (u, k), v in B.items():
            got[(k, u)] = v
        for k in range(9):
            if k not in unk:
                got[(k, k)] = got.get((k, k), 0.0) + 1.0
        want = {(k, u): c0 + c1 * chi for k, u, c0, c1 in gold[side]}
        keys = set(want) | {kk for kk, v in got.items() if abs(v) > 1e-15}
        for key in keys:
            assert abs(got.get(key, 0.0) - want.get(key, 0.0)) < 1e-14, (side, key)
    # top wall, interior x: off-diagonal couplings of Eq. 37
    node = (pr.ny - 1) * pr.nx + 3
    B = _local_block(pr, node, (4, 7, 8))
    for k, u, c0, _ in gold["wall_top_offdiagonal"]:
        assert B[(u, k)] == c0


# ------------------------------------------------------------- invariants --

@pytest.mark.parametrize("q", [9, 19])
def test_uniform_equilibrium_is_a_fixed_point(q):
    nz = 4 if q == 19 else 1
    case = I.periodic_box(6, 5, nz, lattice=q, tau=0.53, cs_smag=0.1)
    pr = O.Problem(case)
    u = np.array([0.03, -0.02, 0.01])[: pr.lat.d]
    p = O.equilibrium(pr.lat, np.full(pr.n, 1.01), np.repeat(u[:, None], pr.n, 1))
    g = pr.g()
    for _ in range(5):
        _, _, p2, _ = pr.step(p, g)
        np.testing.assert_allclose(p2, p, atol=2e-16)
        p = p2


@pytest.mark.parametrize("q", [9, 19])
def test_conservation_in_a_periodic_box(q):
    """Mass is conserved for any design; momentum too when there is no solid."""
    nz = 4 if q == 19 else 1
    shape = (nz, 7, 9)
    gam = np.clip(I.minmax_noise(shape, 1.0, 3), 0, 1)
    for gamma, momentum in ((gam, False), (np.zeros(shape), True)):
        case = I.periodic_box(9, 7, nz, lattice=q, tau=0.52, cs_smag=0.12, gamma=gamma)
        pr = O.Problem(case)
        p = _random_state(pr.lat, pr.n, amp=0.01)
        m0, j0 = p.sum(), pr.lat.c.T @ p.sum(1)
        g = pr.g()
        for _ in range(100):
            _, _, p, _ = pr.step(p, g)
        assert abs(p.sum() - m0) < 1e-11 * m0
        if momentum:
            np.testing.assert_allclose(pr.lat.c.T @ p.sum(1), j0, atol=1e-12)


@pytest.mark.parametrize("q", [9, 19])
def test_shear_wave_decays_at_the_lattice_viscosity(q):
    """Decaying shear wave u_x = U sin(k y): amplitude ~ exp(-nu k^2 t) with
    nu = (tau - 1/2) cs^2 (Eq. 8); Cs = 0 so tau_eff = tau."""
    ny, tau, U, T = 48, 0.8, 1e-3, 300
    nz = 2 if q == 19 else 1
    case = I.periodic_box(2, ny, nz, lattice=q, tau=tau, cs_smag=0.0)
    pr = O.Problem(case)
    yy = (np.arange(pr.n) // pr.nx) % ny
    k = 2 * np.pi / ny
    u = np.zeros((pr.lat.d, pr.n))
    u[0] = U * np.sin(k * yy)
    p = O.equilibrium(pr.lat, np.ones(pr.n), u)
    g = pr.g()
    amps = []
    for t in range(T):
        f, _, p, aux = pr.step(p, g)
        amps.append((aux["u"][0] * np.sin(k * yy)).sum() / (np.sin(k * yy) ** 2).sum())
    nu = (tau - 0.5) * O.CS2
    rate = -np.polyfit(np.arange(50, T), np.log(amps[50:]), 1)[0]
    assert abs(rate / (nu * k * k) - 1) < 2e-3


def test_poiseuille_profile():
    """Pressure-driven channel (Zou-He velocity inlet with the parabola, Zou-He
    pressure outlet, solid walls) relaxes to the Poiseuille parabola, Cs = 0."""
    nx, ny = 48, 17
    case = I.small_channel(nx, ny, tau=0.8, cs_smag=0.0, u_in=0.02, profile="parabolic",
                           outlet=I.OUTLET_P, noise_amp=0.0)
    gamma = np.zeros((1, ny, nx))
    gamma[case.node_class == I.WALL] = 1.0
    case = case.replace(gamma=gamma)
    pr = O.Problem(case)
    p = pr.initial_state()
    g = pr.g()
    for _ in range(4000):
        _, _, p, aux = pr.step(p, g)
    u = aux["u"][0].reshape(ny, nx)[:, nx // 2]
    expect = I.parabolic_profile(ny, 0.02)
    err = np.linalg.norm(u - expect) / np.linalg.norm(expect)
    assert err < 5e-3, err
    # the flow rate is the imposed one
    assert abs(u.sum() / expect.sum() - 1) < 5e-3
    # pressure gradient dp/dx = -8 rho nu u_max / H^2, p = cs^2 rho
    rho = aux["rho"].reshape(ny, nx)[ny // 2]
    dpdx = np.polyfit(np.arange(10, nx - 10), O.CS2 * rho[10:nx - 10], 1)[0]
    nu = (0.8 - 0.5) * O.CS2
    assert abs(dpdx / (-8 * nu * 0.02 / (ny - 1) ** 2) - 1) < 0.03


@pytest.mark.parametrize("q", [9, 19])
def test_objectives_on_a_uniform_stream(q):
    """Closed forms of the four objective integrands (R10) on a uniform stream
    rho = 1, u = u0 e_x through a uniform partial solid: the equilibrium is
    its own collision (Pi^neq = 0), so
      drag (Eq. 44)      sum_a c_xa g (h_abar - h_a) = -2 g rho u0,
      velocity deviation |u - u_ref|^2 = (u0 - u_ref)^2,
      pressure           cs^2 rho = 1/3,
      dissipation        0."""
    u0, uref, g0 = 0.03, 0.01, 0.3
    nx, ny, nz = 7, 5, (4 if q == 19 else 1)
    case = I.periodic_box(nx, ny, nz, lattice=q, gamma=np.full((nz, ny, nx), g0))
    case = case.replace(obj_uref=(uref, 0.0, 0.0))
    pr = O.Problem(case)
    u = np.zeros((pr.lat.d, pr.n))
    u[0] = u0
    p0 = O.equilibrium(pr.lat, np.ones(pr.n), u)
    g = pr.g()
    f, h, _, aux = pr.step(p0, g)
    want = {I.OBJ_DRAG: -2.0 * g * u0, I.OBJ_VELOCITY_DEV: np.full(pr.n, (u0 - uref) ** 2),
            I.OBJ_PRESSURE: np.full(pr.n, 1.0 / 3.0), I.OBJ_DISSIPATION: np.zeros(pr.n)}
    for kind, w in want.items():
        prk = O.Problem(case.replace(obj_kind=kind))
        got = prk.local_objective(f, h, aux, g)
        assert np.allclose(got, w, rtol=1e-12, atol=1e-15), kind


def test_dissipation_objective_is_the_poiseuille_dissipation():
    """In developed Poiseuille flow (Cs = 0, so nu_eff = nu) the dissipation
    integrand equals 2 rho nu S:S = rho nu (du/dy)^2 of the analytic parabola
    u = 4 u_max y (H - y) / H^2 at the mid-channel nodes, to the scheme's
    second-order accuracy."""
    nx, ny, tau, umax = 48, 17, 0.8, 0.02
    case = I.small_channel(nx, ny, tau=tau, cs_smag=0.0, u_in=umax, profile="parabolic",
                           outlet=I.OUTLET_P, noise_amp=0.0, obj_kind=I.OBJ_DISSIPATION)
    gamma = np.zeros((1, ny, nx))
    gamma[case.node_class == I.WALL] = 1.0
    case = case.replace(gamma=gamma)
    pr = O.Problem(case)
    p = pr.initial_state()
    g = pr.g()
    for _ in range(4000):
        f, h, p, aux = pr.step(p, g)
    psi = pr.local_objective(f, h, aux, g).reshape(ny, nx)[:, nx // 2]
    H = ny - 1
    y = np.arange(ny)
    nu = (tau - 0.5) / 3.0
    want = nu * (4 * umax * (H - 2 * y) / H ** 2) ** 2
    inner = slice(2, ny - 2)                        # away from the wall rows and their neighbours
    # 2%: the developed profile itself is within 0.5% of the parabola at H = 16 (test_poiseuille_profile), and
    # (du/dy)^2 doubles that; a dropped factor of the integrand (2, tau_eff, rho) would be off by 50-100%
    assert np.abs(psi[inner] - want[inner]).max() <= 0.02 * want[inner].max()
    assert abs(psi[inner].sum() / want[inner].sum() - 1) < 0.02


def test_mirror_symmetry():
    """A y-symmetric channel stays symmetric: rho even, u_x even, u_y odd."""
    nx, ny = 20, 11
    case = I.small_channel(nx, ny, u_in=0.05, profile="parabolic", outlet=I.OUTLET_P)
    gam = case.gamma.copy()
    gam = 0.5 * (gam + gam[:, ::-1, :])
    case = case.replace(gamma=gam)
    pr = O.Problem(case)
    p = pr.initial_state()
    g = pr.g()
    for _ in range(100):
        _, _, p, aux = pr.step(p, g)
    rho = aux["rho"].reshape(ny, nx)
    u = aux["u"].reshape(2, ny, nx)
    np.testing.assert_allclose(rho, rho[::-1], atol=1e-13)
    np.testing.assert_allclose(u[0], u[0][::-1], atol=1e-13)
    np.testing.assert_allclose(u[1], -u[1][::-1], atol=1e-13)


def test_window_criterion():
    """Eq. 26 on numbers worked by hand."""
    r, c = O.criterion(2.0, 1.999, 1e-3)
    assert abs(r - 0.0005) < 1e-15 and c
    r, c = O.criterion(-0.5, -0.4, 1e-3)
    assert abs(r - 0.2) < 1e-15 and not c
    r, c = O.criterion(0.0, 1e-40, 1e-30)
    assert r == 1e-40 and c


# ---------------------------------------------------------------- adjoint --

ADJ_CASES = [
    ("diss-zouhe", lambda: I.small_channel(10, 7, obj_kind=I.OBJ_DISSIPATION, window_len=8,
                                            outlet=I.OUTLET_P, profile="parabolic")),
    ("veldev-zg", lambda: I.small_channel(10, 7, obj_kind=I.OBJ_VELOCITY_DEV, window_len=8,
                                           outlet=I.OUTLET_ZG, sample_every=2)),
    ("pressure", lambda: I.small_channel(9, 6, obj_kind=I.OBJ_PRESSURE, window_len=6)),
    ("drag-periodic", lambda: I.small_channel(9, 6, obj_kind=I.OBJ_DRAG, window_len=6,
                                               periodic_x=True, g_max=0.9)),
    ("d3q19-duct", lambda: I.small_duct3d(6, 5, 5, window_len=5)),
    ("d3q19-diss", lambda: I.small_duct3d(6, 5, 4, window_len=4, obj_kind=I.OBJ_DISSIPATION,
                                          periodic_z=True)),
]


def _developed_start(pr, steps=30):
    from _util import initial_flow
    p = initial_flow(pr)
    g = pr.g()
    for _ in range(steps):
        _, _, p, _ = pr.step(p, g)
    return p


@pytest.mark.parametrize("name,mk", ADJ_CASES, ids=[c[0] for c in ADJ_CASES])
def test_adjoint_matches_complex_step(name, mk):
    """<dJ/dgamma, d> equals the complex-step derivative of the oracle's own
    forward window (exact to rounding), in a random direction d; likewise for
    the adjoint of the window's start field.  Pins Eqs. 30-40 including every
    boundary transpose, the sampling weights and the objective sources."""
    case = mk()
    pr = O.Problem(case)
    p0 = _developed_start(pr)
    rng = np.random.default_rng(5)
    traj = pr.run_window(p0)[3]
    _, dgamma, a0 = pr.adjoint_window(traj)
    d = rng.standard_normal(pr.n)
    h = 1e-30
    J_c = pr.window_objective(p0.astype(complex), case.gamma.reshape(-1) + 1j * h * d)
    want = J_c.imag / h
    got = dgamma @ d
    assert abs(want) > 1e-12                      # a non-degenerate direction
    assert abs(got - want) <= 1e-10 * abs(want), (got, want)
    dp = rng.standard_normal(p0.shape) * pr.lat.w[:, None]
    J_c = pr.window_objective(p0 + 1j * h * dp, case.gamma.reshape(-1))
    want = J_c.imag / h
    got = (a0 * dp).sum()
    assert abs(got - want) <= 1e-10 * abs(want), (got, want)


def test_adjoint_matches_central_differences():
    """Single-node perturbations of gamma (the protocol of Sec. 4.2.1): central
    differences with h = 1e-6 agree with the adjoint to 1e-6 relative."""
    case = I.small_channel(12, 8, obj_kind=I.OBJ_DISSIPATION, window_len=10)
    pr = O.Problem(case)
    p0 = _developed_start(pr, 40)
    traj = pr.run_window(p0)[3]
    _, dgamma, _ = pr.adjoint_window(traj)
    gam = case.gamma.reshape(-1)
    for node in (3 * 12 + 4, 4 * 12 + 7, 2 * 12 + 9):
        e = np.zeros(pr.n)
        e[node] = 1e-6
        fd = (pr.window_objective(p0, gam + e) - pr.window_objective(p0, gam - e)) / 2e-6
        assert abs(fd - dgamma[node]) <= 1e-6 * abs(dgamma[node]), (node, fd, dgamma[node])


@pytest.mark.parametrize("q,outlet", [(9, I.OUTLET_P), (9, I.OUTLET_ZG), (19, I.OUTLET_ZG)])
def test_uniform_flow_is_a_fixed_point_of_inlet_and_outlet(q, outlet):
    """A uniform stream u0 e_x at rho = 1 through a domain periodic across the
    flow is an exact fixed point: the Zou-He rules reproduce rho = 1 and u0
    (Eqs. 20-21), the moving-wall inlet reproduces the odd part of the
    equilibrium, 2 w_a rho c_a.u / cs^2, and the zero-gradient outlet copies a
    uniform field."""
    u0 = 0.04
    nx, ny, nz = 9, 5, (4 if q == 19 else 1)
    cls = np.zeros((nz, ny, nx), np.uint8)
    cls[:, :, 0] = I.INLET
    cls[:, :, nx - 1] = outlet
    case = I.Case(name="stream", lattice=q, nx=nx, ny=ny, nz=nz, tau=0.56, cs_smag=0.1,
                  node_class=cls, gamma=np.zeros((nz, ny, nx)), inlet_u=np.full((nz, ny), u0),
                  obj_weights=np.zeros((nz, ny, nx)), periodic=(0, 1, 1 if q == 19 else 0),
                  design_box=(0, nx, 0, ny, 0, nz))
    pr = O.Problem(case)
    u = np.zeros((pr.lat.d, pr.n))
    u[0] = u0
    p = O.equilibrium(pr.lat, np.ones(pr.n), u)
    g = pr.g()
    for _ in range(3):
        _, _, p2, _ = pr.step(p, g)
        np.testing.assert_allclose(p2, p, atol=3e-17)
        p = p2


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("window_len,sample_every,sample_from", [(12, 1, 0), (12, 3, 0), (12, 3, 3), (20, 4, 8)])
def test_window_means_and_drag_coefficient_in_closed_form(q, window_len, sample_every, sample_from):
    """Eq. 25 (C_d = F_x / (1/2 rho_0 U^2 L)) and the window means of Eq. 42
    (samples every dW-th step from the first sampled step, weight dW over the
    sampled span) on a decaying uniform stream whose every sample is known in
    closed form.  A dropped 1/2, a squared L, a wrong sample count or shifted
    sampling instants each change the result by far more than rounding."""
    from _util import decaying_stream_window
    J, M, J_want, M_want = decaying_stream_window(q, window_len, sample_every, sample_from)
    assert abs(J - J_want) <= 1e-13 * abs(J_want), (J, J_want)
    assert abs(M - M_want) <= 1e-13 * abs(M_want), (M, M_want)
