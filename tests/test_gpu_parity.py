"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances (from the arithmetic):
  * FP64 build vs oracle: 1e-12 relative (norm-wise) on states, window means,
    gradients -- both sides are FP64 and the trajectories are non-chaotic over
    these horizons, so differences are rounding-order only;
  * FP32 build after 200 steps: 1e-5 relative (norm-wise) on rho and on u over
    fluid nodes (gamma < 1/2);
  * FP32 adjoint over short windows: gradient cosine >= 0.9999 and 1e-3
    relative norm-wise against the FP64 oracle.
Sizes span several 128-node row tiles with a ragged tail.
"""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2608_19617_b300 import binding as B
from paper_2608_19617_b300 import inputs as I

from _util import cosine, f32_inputs, fluid_moments, initial_flow, oracle_advance, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2608_19617_b300 import build
    build.build()
    B.lib()


FWD_CASES = {
    "zouhe300x20": lambda: I.small_channel(300, 20, outlet=I.OUTLET_P, profile="parabolic", u_in=0.06,
                                           tau=0.53, cs_smag=0.12, window_len=20),
    "zerograd140x13": lambda: I.small_channel(140, 13, outlet=I.OUTLET_ZG, u_in=0.05, tau=0.52,
                                              window_len=20, obj_kind=I.OBJ_VELOCITY_DEV),
    "periodic-x131x9": lambda: I.small_channel(131, 9, periodic_x=True, tau=0.55, window_len=20,
                                               obj_kind=I.OBJ_DRAG, g_max=0.8),
    "duct3d-150x7x6": lambda: I.small_duct3d(150, 7, 6, tau=0.53, window_len=20),
    "duct3d-periodicz": lambda: I.small_duct3d(133, 6, 5, tau=0.54, periodic_z=True, window_len=20,
                                               obj_kind=I.OBJ_DISSIPATION),
    # the layout of the U-bend workloads at reduced size: a velocity inlet and
    # a zero-gradient outlet side by side on the x = 0 face, walls and 3D wall
    # corners around them, the bend near x = nx-1
    "ubend48x28x16": lambda: I.ubend_case(48, 28, 16, 8, tau=0.52, cs_smag=0.1, window_len=20, ckpt_every=20,
                                          ckpt_format=I.CKPT_NATIVE),
}


def _developed(pr, steps):
    return oracle_advance(pr, initial_flow(pr), steps)


@pytest.mark.parametrize("name", list(FWD_CASES))
def test_forward_fp64_matches_oracle(name):
    case = f32_inputs(FWD_CASES[name]())
    pr = O.Problem(case)
    sol = B.Solver(case, B.LBM_FP64)
    sol.advance(200)
    got = sol.get_state()
    want = oracle_advance(pr, pr.initial_state(), 200)
    assert rel_err(got, want) < 1e-12
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("name", list(FWD_CASES))
def test_forward_fp32_within_1e5(name):
    case = f32_inputs(FWD_CASES[name]())
    pr = O.Problem(case)
    sol = B.Solver(case, B.LBM_FP32)
    sol.advance(200)
    got = sol.get_state()
    want = oracle_advance(pr, pr.initial_state(), 200)
    rg, ug = fluid_moments(pr, got, case)
    rw, uw = fluid_moments(pr, want, case)
    assert rel_err(rg, rw) < 1e-5
    assert rel_err(ug, uw) < 1e-5


def _periodic_y_channel(nx, ny, **kw):
    """A 2D channel periodic in y (no walls along x): inlet on x = 0; on
    x = nx-1 a zero-gradient outlet on rows 0-2 and walls on the other rows.
    The outlet node on row 0 copies a population of the wall node on row
    ny-1 across the periodic wrap, so the adjoint must pull it back there."""
    c = I.small_channel(nx, ny, outlet=I.OUTLET_ZG, **kw)
    cls = np.zeros_like(c.node_class)
    cls[0, :, 0] = I.INLET
    cls[0, :, nx - 1] = I.WALL
    cls[0, 0:3, nx - 1] = I.OUTLET_ZG
    gamma = c.gamma.copy()
    gamma[0, 0, :] = gamma[0, 2, :]
    gamma[0, ny - 1, :] = gamma[0, ny - 3, :]
    gamma[cls == I.INLET] = 0.0
    gamma[cls == I.OUTLET_ZG] = 0.0
    gamma[cls == I.WALL] = 1.0
    w = np.zeros_like(c.obj_weights)
    w[0, :, nx - 4] = 1.0 / ny     # near the outlet, so that the adjoint window reaches it
    return c.replace(name=f"channel{nx}x{ny}-periodic-y", node_class=cls, gamma=gamma,
                     inlet_u=np.full((1, ny), 0.05), obj_weights=w, periodic=(0, 1, 0),
                     design_box=(1, nx - 1, 0, ny, 0, 1))


ADJ_CASES = {
    "diss-zouhe": lambda: I.small_channel(150, 12, obj_kind=I.OBJ_DISSIPATION, window_len=12,
                                          outlet=I.OUTLET_P, profile="parabolic", tau=0.53, cs_smag=0.12),
    "veldev-zg-dw3": lambda: I.small_channel(140, 11, obj_kind=I.OBJ_VELOCITY_DEV, window_len=12,
                                             outlet=I.OUTLET_ZG, sample_every=3, tau=0.52),
    "pressure": lambda: I.small_channel(133, 10, obj_kind=I.OBJ_PRESSURE, window_len=10, tau=0.56),
    "veldev-zg-periodic-y": lambda: _periodic_y_channel(137, 9, obj_kind=I.OBJ_VELOCITY_DEV, window_len=12,
                                                        sample_every=3, tau=0.53),
    "drag-periodic": lambda: I.small_channel(129, 9, obj_kind=I.OBJ_DRAG, window_len=10,
                                             periodic_x=True, g_max=0.9, monitor_kind=I.MON_OBJECTIVE),
    "d3q19-pressure": lambda: I.small_duct3d(130, 6, 6, window_len=8, tau=0.53),
    "d3q19-diss-periodicz": lambda: I.small_duct3d(131, 6, 5, window_len=8, obj_kind=I.OBJ_DISSIPATION,
                                                   periodic_z=True, tau=0.54),
    # pressure drop between the legs at x = 8: a 12-step adjoint reaches the
    # transposed inlet and zero-gradient rules on the x = 0 face; the design
    # box spans the whole duct so that the gradient sees them
    # the smallest bounded lattices (one interior node) and a single inner row
    # with a ragged tail
    "smallest-2d-3x3": lambda: I.small_channel(3, 3, obj_kind=I.OBJ_DISSIPATION, window_len=6, ckpt_every=2,
                                               tau=0.56),
    "smallest-3d-3x3x3": lambda: I.small_duct3d(3, 3, 3, obj_kind=I.OBJ_DISSIPATION, window_len=6, ckpt_every=2,
                                                tau=0.56),
    "one-inner-row-130x3": lambda: I.small_channel(130, 3, outlet=I.OUTLET_ZG, obj_kind=I.OBJ_VELOCITY_DEV,
                                                   window_len=8, ckpt_every=4, tau=0.53),
    "ubend48x28x16-pressure": lambda: I.ubend_case(48, 28, 16, 8, tau=0.52, cs_smag=0.1, window_len=12,
                                                   ckpt_every=4, ckpt_format=I.CKPT_NATIVE).replace(
                                                       design_box=(1, 47, 1, 27, 1, 15)),
}


def _gpu_window_and_adjoint(case, precision, p_start, **kw):
    sol = B.Solver(case, precision, **kw)
    sol.set_state(p_start)
    J, M = sol.step_window()
    Jeff = sol.adjoint_window()
    grad = sol.design_gradient()
    a0 = sol.get_adjoint_state()
    return sol, J, M, Jeff, grad, a0


@pytest.mark.parametrize("name", list(ADJ_CASES))
def test_window_and_adjoint_fp64_match_oracle(name):
    case = f32_inputs(ADJ_CASES[name]())
    pr = O.Problem(case)
    p0 = _developed(pr, 40)
    _, Jw, Mw, traj = pr.run_window(p0)
    _, grad_w, a0_w = pr.adjoint_window(traj)
    sol, J, M, Jeff, grad, a0 = _gpu_window_and_adjoint(case, B.LBM_FP64, p0)
    assert abs(J - Jw) <= 1e-12 * abs(Jw)
    assert abs(M - Mw) <= 1e-12 * abs(Mw) + 1e-300
    assert Jeff == J
    dbox = np.zeros((case.nz, case.ny, case.nx), bool)
    x0, x1, y0, y1, z0, z1 = case.design_box
    dbox[z0:z1, y0:y1, x0:x1] = True
    dbox = dbox.reshape(-1)
    assert rel_err(grad[dbox], grad_w[dbox]) < 1e-11
    assert np.all(grad[~dbox] == 0)
    assert rel_err(a0, a0_w) < 1e-11


@pytest.mark.parametrize("name", list(ADJ_CASES))
def test_window_and_adjoint_fp32_match_oracle(name):
    case = f32_inputs(ADJ_CASES[name]())
    pr = O.Problem(case)
    p0 = _developed(pr, 40)
    _, Jw, Mw, traj = pr.run_window(p0)
    _, grad_w, a0_w = pr.adjoint_window(traj)
    sol, J, M, Jeff, grad, a0 = _gpu_window_and_adjoint(case, B.LBM_FP32, p0)
    assert abs(J - Jw) <= 1e-4 * abs(Jw)
    x0, x1, y0, y1, z0, z1 = case.design_box
    m = np.zeros((case.nz, case.ny, case.nx), bool)
    m[z0:z1, y0:y1, x0:x1] = True
    m = m.reshape(-1)
    assert cosine(grad[m], grad_w[m]) > 0.9999
    assert rel_err(grad[m], grad_w[m]) < 1e-3
    assert cosine(a0, a0_w) > 0.9999


# Windows whose only sample is taken on f^{n0}, pulled from the fixed start
# field: |W| = 1, and dW = |W|.
DESIGN_FREE_WINDOWS = {
    "single-step-window": lambda: I.small_channel(133, 10, obj_kind=I.OBJ_PRESSURE, window_len=1, ckpt_every=1,
                                                  tau=0.56),
    "one-sample-per-window": lambda: I.small_duct3d(131, 6, 6, window_len=6, sample_every=6, ckpt_every=3,
                                                    tau=0.53),
}


@pytest.mark.parametrize("name", list(DESIGN_FREE_WINDOWS))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_windows_whose_sample_precedes_the_design(name, precision):
    """The window's only sample is taken on the field pulled from the fixed
    start field (Eq. 42 with samples at n0, n0 + dW, ...), so J does not
    depend on the design: the oracle's gradient and the GPU's are exactly
    zero, and the start-field adjoint is the sample's own source."""
    case = f32_inputs(DESIGN_FREE_WINDOWS[name]())
    pr = O.Problem(case)
    p0 = _developed(pr, 40)
    _, Jw, _, traj = pr.run_window(p0)
    _, grad_w, a0_w = pr.adjoint_window(traj)
    assert np.all(grad_w == 0) and np.count_nonzero(a0_w) > 0
    prec = B.LBM_FP64 if precision == "fp64" else B.LBM_FP32
    _, J, _, Jeff, grad, a0 = _gpu_window_and_adjoint(case, prec, p0)
    assert np.all(grad == 0)
    assert abs(J - Jw) <= (1e-12 if precision == "fp64" else 1e-5) * abs(Jw)
    assert rel_err(a0, a0_w) < (1e-11 if precision == "fp64" else 1e-5)


def test_zero_objective_weights():
    """No objective weights: J is exactly 0, the adjoint sweep carries exact
    zeros (start-field adjoint and gradient), and the window's monitor is the
    oracle's."""
    case = f32_inputs(I.small_duct3d(131, 6, 5, window_len=8, ckpt_every=4, tau=0.53))
    case = case.replace(obj_weights=np.zeros_like(case.obj_weights))
    pr = O.Problem(case)
    p0 = _developed(pr, 30)
    _, Jw, Mw, _ = pr.run_window(p0)
    _, J, M, Jeff, grad, a0 = _gpu_window_and_adjoint(case, B.LBM_FP64, p0)
    assert Jw == 0 and J == 0 and Jeff == 0
    assert np.all(grad == 0) and np.all(a0 == 0)
    assert abs(M - Mw) <= 1e-12 * abs(Mw)


def test_empty_design_box():
    """An empty design box: the gradient is exactly zero everywhere, while J,
    the monitor and the start-field adjoint are the oracle's."""
    case = f32_inputs(I.small_channel(140, 11, obj_kind=I.OBJ_VELOCITY_DEV, window_len=12, ckpt_every=4,
                                      outlet=I.OUTLET_ZG, tau=0.52)).replace(design_box=(5, 5, 0, 0, 0, 0))
    pr = O.Problem(case)
    p0 = _developed(pr, 40)
    _, Jw, Mw, traj = pr.run_window(p0)
    _, _, a0_w = pr.adjoint_window(traj)
    _, J, M, _, grad, a0 = _gpu_window_and_adjoint(case, B.LBM_FP64, p0)
    assert np.all(grad == 0)
    assert abs(J - Jw) <= 1e-12 * abs(Jw) and abs(M - Mw) <= 1e-12 * abs(Mw)
    assert rel_err(a0, a0_w) < 1e-11


def test_recompute_from_checkpoints_is_bitwise():
    """Segments of K < |W| recompute the same trajectory: the adjoint field is
    bitwise identical; the gradient differs only by the order in which the
    per-segment FP32 partials are folded into the FP64 sums."""
    case = f32_inputs(I.small_channel(150, 12, window_len=24, outlet=I.OUTLET_P, tau=0.53))
    pr = O.Problem(case)
    p0 = _developed(pr, 30)
    grads, adj = [], []
    for K in (24, 6, 1):
        sol = B.Solver(case.replace(ckpt_every=K), B.LBM_FP32)
        sol.set_state(p0)
        sol.step_window()
        sol.adjoint_window()
        grads.append(sol.design_gradient())
        adj.append(sol.get_adjoint_state())
    assert np.array_equal(adj[0], adj[1]) and np.array_equal(adj[0], adj[2])
    assert rel_err(grads[1], grads[0]) < 1e-6 and rel_err(grads[2], grads[0]) < 1e-6


@pytest.mark.parametrize("fmt", [I.CKPT_FP16, I.CKPT_BF16])
def test_sixteen_bit_checkpoints_keep_the_gradient(fmt):
    case = f32_inputs(I.small_channel(200, 16, window_len=40, outlet=I.OUTLET_P, tau=0.53))
    pr = O.Problem(case)
    p0 = _developed(pr, 60)
    out = {}
    for f in (I.CKPT_NATIVE, fmt):
        sol = B.Solver(case.replace(ckpt_every=8, ckpt_format=f), B.LBM_FP32)
        sol.set_state(p0)
        J, _ = sol.step_window()
        sol.adjoint_window()
        out[f] = (J, sol.design_gradient())
    assert out[fmt][0] == out[I.CKPT_NATIVE][0]     # the forward is not touched
    assert cosine(out[fmt][1], out[I.CKPT_NATIVE][1]) > 0.999


def test_window_sequence_and_criterion_fp64():
    """Consecutive windows: means and the ratio of Eq. 26 against the oracle."""
    case = f32_inputs(I.small_channel(140, 12, window_len=15, outlet=I.OUTLET_P, tau=0.53))
    pr = O.Problem(case)
    rec = pr.run_until_converged(max_windows=4)
    sol = B.Solver(case, B.LBM_FP64)
    for i, r in enumerate(rec):
        J, M = sol.step_window()
        conv, ratio = sol.window_converged()
        assert abs(J - r["J"]) <= 1e-12 * abs(r["J"])
        assert abs(M - r["M"]) <= 1e-12 * abs(r["M"])
        if i == 0:
            assert ratio == float("inf") and not conv
        else:
            assert abs(ratio - r["ratio"]) <= 1e-9 * abs(r["ratio"]) + 1e-15
            assert conv == r["converged"]


def test_error_paths():
    case = f32_inputs(I.small_channel(64, 10, window_len=10))
    sol = B.Solver(case, B.LBM_FP32)
    with pytest.raises(B.LbmError) as e:
        sol.adjoint_window()
    assert e.value.status == B.LBM_ERR_STATE
    with pytest.raises(B.LbmError) as e:
        sol.design_gradient()
    assert e.value.status == B.LBM_ERR_STATE
    p = sol.get_state()
    bad = p.copy()
    bad[0, 5] = np.nan
    with pytest.raises(B.LbmError) as e:
        sol.set_state(bad)
    assert e.value.status == B.LBM_ERR_ARG
    neg = p.copy()
    for yy in (3, 4, 5):                             # a 3x3 block: its centre pulls rho < 0
        neg[:, yy * 64 + 19:yy * 64 + 22] = -0.2
    sol.set_state(neg)
    with pytest.raises(B.LbmError) as e:
        sol.step_window()
    assert e.value.status == B.LBM_ERR_NONFINITE
    sol.set_state(p)                                 # recovers
    sol.step_window()
    with pytest.raises(B.LbmError) as e:
        sol.set_design(np.full(case.n, 1.5, np.float32))
    assert e.value.status == B.LBM_ERR_ARG


def test_state_round_trip_and_counters():
    case = f32_inputs(I.small_duct3d(20, 6, 6))
    sol = B.Solver(case, B.LBM_FP64)
    rng = np.random.default_rng(0)
    lat = O.Lattice(19)
    p = lat.w[:, None] * (1 + 0.01 * rng.standard_normal((19, case.n)))
    sol.set_state(p)
    assert np.abs(sol.get_state() - p).max() < 1e-16
    sol.advance(3)
    assert sol.counters() == (3, 0)


def test_device_buffers_and_autograd():
    """Design and gradient through device pointers, and the autograd function."""
    import torch
    from paper_2608_19617_b300.autograd import window_objective
    case = f32_inputs(I.small_channel(140, 12, window_len=12, outlet=I.OUTLET_P, tau=0.53))
    pr = O.Problem(case)
    sol = B.Solver(case, B.LBM_FP64)
    gam = torch.tensor(case.gamma.reshape(-1), dtype=torch.float32, device="cuda", requires_grad=True)
    J = window_objective(gam, sol, 2)
    J.backward()
    rec = pr.run_until_converged(max_windows=2)
    traj = pr.run_window(rec[-1]["p_start"])[3]
    _, grad_w, _ = pr.adjoint_window(traj)
    assert abs(J.item() - rec[-1]["J"]) <= 1e-12 * abs(rec[-1]["J"])
    x0, x1, y0, y1, _, _ = case.design_box
    m = np.zeros((case.ny, case.nx), bool)
    m[y0:y1, x0:x1] = True
    g = gam.grad.detach().cpu().numpy().astype(np.float64)
    assert rel_err(g[m.reshape(-1)], grad_w[m.reshape(-1)]) < 1e-6   # float32 gradient tensor


# ---------------------------------------------------------------------------
# Full-size workloads in the benchmark's launch configuration.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["wake1024x256", "step2048x512", "ubend256x128x64"])
def test_full_size_one_step_against_oracle(name):
    """After a spin-up on the GPU, one more GPU step equals the oracle's step
    from the same field, element by element (FP32 vs FP64)."""
    case = f32_inputs(I.WORKLOADS[name]())
    sol = B.Solver(case, B.LBM_FP32)
    sol.advance(300)
    p = sol.get_state()
    sol.advance(1)
    got = sol.get_state()
    pr = O.Problem(case)
    want = oracle_advance(pr, p, 1)
    assert np.abs(got - want).max() < 2e-6


def _x_crop(case, x0, x1):
    """Columns x0 .. x1-1 of a lattice as a lattice of its own, the cut faces
    made walls.  One step of a node at least one column away from a cut pulls
    the same populations as in the whole lattice."""
    cls = case.node_class[:, :, x0:x1].copy()
    if x0 > 0:
        cls[:, :, 0] = I.WALL
    if x1 < case.nx:
        cls[:, :, -1] = I.WALL
    uin = case.inlet_u if x0 == 0 else np.zeros_like(case.inlet_u)
    return case.replace(name=f"{case.name}[x{x0}:{x1}]", nx=x1 - x0, node_class=cls,
                        gamma=case.gamma[:, :, x0:x1].copy(), inlet_u=uin,
                        obj_weights=case.obj_weights[:, :, x0:x1].copy(),
                        design_box=(1, x1 - x0 - 1, 1, case.ny - 1, 1, case.nz - 1))


def test_default_workload_one_step_against_oracle_on_crops():
    """The 384x192x192 U-bend (the benchmark's default workload): after a
    spin-up, one GPU step over the whole lattice in the benchmark's launch
    configuration equals, element by element, the oracle's step on two
    64-column crops of the same field -- the x = 0 end (velocity inlet and
    zero-gradient outlet side by side, the legs) and the far end (the bend) --
    at every node but the crops' cut faces."""
    case = f32_inputs(I.WORKLOADS["ubend384x192x192"]()).replace(window_len=20, ckpt_every=10)
    sol = B.Solver(case, B.LBM_FP32)
    sol.advance(300)
    q, nx, ny, nz = case.lattice, case.nx, case.ny, case.nz
    p = sol.get_state().reshape(q, nz, ny, nx)
    sol.advance(1)
    got = sol.get_state().reshape(q, nz, ny, nx)
    sol.close()
    for x0, x1 in ((0, 64), (320, 384)):
        crop = _x_crop(case, x0, x1)
        want = oracle_advance(O.Problem(crop), p[:, :, :, x0:x1].reshape(q, -1), 1).reshape(q, nz, ny, x1 - x0)
        lo, hi = (1 if x0 > 0 else 0), (x1 - x0 - 1 if x1 < nx else x1 - x0)
        diff = np.abs(got[:, :, :, x0 + lo:x0 + hi] - want[:, :, :, lo:hi])
        assert diff.max() < 2e-6, (x0, x1, float(diff.max()))


# Columns around each objective plane: ubend256 and ubend384 sample the
# pressure drop on x = 32 / 48, step2048x512 on x = 8 and x = nx - 9.
FULL_SIZE_ADJOINT_CROPS = {
    "ubend256x128x64": [(26, 38)],
    "ubend384x192x192": [(42, 54)],
    "step2048x512": [(0, 14), (2034, 2048)],
}


@pytest.mark.parametrize("name", list(FULL_SIZE_ADJOINT_CROPS))
def test_full_size_two_step_adjoint_against_oracle_on_crops(name):
    """A workload at full size in the benchmark's launch configuration (its
    own checkpoint format), design box widened to the whole lattice: a
    two-step window and its adjoint over the whole lattice, against the
    oracle's on 12-14 columns around each objective plane.  In two steps the
    adjoint of a plane's samples reaches two columns to each side, so the
    gradient and the start-field adjoint of the columns away from the cuts are
    those of the whole lattice, J is the sum of the crops' (it is linear in
    the plane weights), and the gradient is exactly zero beyond that reach.
    The spin-up (5000 steps) brings flow to every plane: the sensitivity
    -6 m.A1 vanishes where the fluid is still at rest.  The recompute starts
    from the window's checkpoint, stored in the workload's format: a BF16
    deviation keeps 8 significant bits (rounding 2^-9 of itself), FP16 11, so
    the gradient bound is 5e-3 with BF16 and 1e-3 otherwise."""
    case = f32_inputs(I.WORKLOADS[name]())
    tol = 5e-3 if case.ckpt_format == I.CKPT_BF16 else 1e-3
    q, nx, ny, nz = case.lattice, case.nx, case.ny, case.nz
    z0, z1 = (1, nz - 1) if q == 19 else (0, 1)
    case = case.replace(window_len=2, ckpt_every=2, design_box=(1, nx - 1, 1, ny - 1, z0, z1))
    sol = B.Solver(case, B.LBM_FP32)
    sol.advance(5000)
    p0 = sol.get_state().reshape(q, nz, ny, nx)
    J, _ = sol.step_window()
    sol.adjoint_window()
    grad = sol.design_gradient().reshape(nz, ny, nx)
    a0 = sol.get_adjoint_state().reshape(q, nz, ny, nx)
    sol.close()
    J_crops = 0.0
    reach = np.zeros(nx, bool)
    for x0, x1 in FULL_SIZE_ADJOINT_CROPS[name]:
        crop = _x_crop(case, x0, x1)
        pr = O.Problem(crop)
        _, Jw, _, traj = pr.run_window(p0[:, :, :, x0:x1].reshape(q, -1))
        _, grad_w, a0_w = pr.adjoint_window(traj)
        J_crops += Jw
        lo, hi = (1 if x0 > 0 else 0), (x1 - x0 - 1 if x1 < nx else x1 - x0)
        g, gw = grad[:, :, x0 + lo:x0 + hi], grad_w.reshape(nz, ny, x1 - x0)[:, :, lo:hi]
        a, aw = a0[:, :, :, x0 + lo:x0 + hi], a0_w.reshape(q, nz, ny, x1 - x0)[:, :, :, lo:hi]
        assert np.count_nonzero(gw) > 0 and np.count_nonzero(aw) > 0
        assert cosine(g, gw) > 0.9999 and rel_err(g, gw) < tol, (x0, x1, cosine(g, gw), rel_err(g, gw))
        assert cosine(a, aw) > 0.9999 and rel_err(a, aw) < tol, (x0, x1, cosine(a, aw), rel_err(a, aw))
        reach[x0 + 2:x1 - 2] = True
    assert abs(J - J_crops) <= 1e-4 * abs(J_crops)
    assert np.all(grad[:, :, ~reach] == 0)


def test_channel_workload_fp64_at_full_size_against_oracle():
    """The 128x64 channel workload (parabolic Zou-He inlet, zero-gradient
    outlet, disk plus noise, FP64): 200 steps from rest against the oracle,
    1e-12 relative; then a window of its full length (200 steps, K = 200) and
    its adjoint, window means 1e-12 and gradient 1e-11."""
    case = f32_inputs(I.WORKLOADS["channel128x64"]())
    pr = O.Problem(case)
    sol = B.Solver(case, B.LBM_FP64)
    sol.advance(200)
    got = sol.get_state()
    want = oracle_advance(pr, pr.initial_state(), 200)
    assert rel_err(got, want) < 1e-12
    sol.set_state(want)
    J, M = sol.step_window()
    sol.adjoint_window()
    grad = sol.design_gradient()
    _, Jw, Mw, traj = pr.run_window(want)
    _, grad_w, _ = pr.adjoint_window(traj)
    assert abs(J - Jw) <= 1e-12 * abs(Jw)
    assert abs(M - Mw) <= 1e-12 * abs(Mw)
    x0, x1, y0, y1, z0, z1 = case.design_box
    m = np.zeros((case.nz, case.ny, case.nx), bool)
    m[z0:z1, y0:y1, x0:x1] = True
    m = m.reshape(-1)
    assert rel_err(grad[m], grad_w[m]) < 1e-11


def test_full_size_short_window_adjoint_against_oracle():
    """A two-step window at the wake workload's full size: gradient and start
    adjoint against the oracle (FP32 vs FP64)."""
    import numpy as np
    base = I.WORKLOADS["wake1024x256"]()
    # drag of the partial bounce-back force summed over the whole lattice, so
    # that a two-step adjoint reaches every design node
    case = f32_inputs(base.replace(obj_kind=I.OBJ_DRAG, obj_weights=np.ones_like(base.obj_weights),
                                   window_len=2, ckpt_every=2))
    sol = B.Solver(case, B.LBM_FP32)
    sol.advance(3000)                               # let the wake reach the design box
    p = sol.get_state()
    sol.step_window()
    sol.adjoint_window()
    grad = sol.design_gradient()
    pr = O.Problem(case)
    _, _, _, traj = pr.run_window(p)
    _, grad_w, _ = pr.adjoint_window(traj)
    x0, x1, y0, y1, _, _ = case.design_box
    m = np.zeros((case.ny, case.nx), bool)
    m[y0:y1, x0:x1] = True
    m = m.reshape(-1)
    assert np.abs(grad_w[m]).max() > 0
    assert np.all(grad[~m] == 0)
    assert cosine(grad[m], grad_w[m]) > 0.9999


def test_phase_timing_under_graphs():
    """Timing events recorded inside replayed graphs are readable and leave no
    error behind for the next call."""
    case = f32_inputs(I.small_channel(150, 12, window_len=20, ckpt_every=5, outlet=I.OUTLET_P, tau=0.53))
    sol = B.Solver(case, B.LBM_FP32)
    sol.set_timing(True)
    for _ in range(2):
        sol.step_window()
        sol.adjoint_window()
        sol.design_gradient()
    t = sol.get_timing()
    assert t["forward"]["launches"] == 40 and t["adjoint"]["launches"] == 40
    assert t["recompute"]["launches"] == 2 * 4 * 4
    assert all(t[k]["ms"] > 0 for k in ("forward", "recompute", "adjoint"))


def test_graph_replay_matches_direct_launches():
    """Windows and sweeps replayed as CUDA graphs give bitwise the results of
    individually launched kernels, including an odd |W| (parity flips)."""
    case = f32_inputs(I.small_channel(150, 12, window_len=15, ckpt_every=5, outlet=I.OUTLET_P, tau=0.53))
    out = []
    for graphs in (False, True):
        sol = B.Solver(case, B.LBM_FP32)
        sol.set_graphs(graphs)
        rec = [sol.step_window() for _ in range(3)]
        sol.adjoint_window()
        out.append((rec, sol.design_gradient(), sol.get_state()))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


def test_programmatic_dependent_launch_matches():
    """Step kernels launched with programmatic dependent launch (graphs on and
    off) give bitwise the results of plain launches."""
    case = f32_inputs(I.small_duct3d(140, 7, 6, window_len=12, ckpt_every=4, tau=0.53))
    out = []
    for pdl, graphs in ((False, True), (True, True), (True, False)):
        sol = B.Solver(case, B.LBM_FP32)
        sol.set_pdl(pdl)
        sol.set_graphs(graphs)
        rec = [sol.step_window() for _ in range(2)]
        sol.adjoint_window()
        out.append((rec, sol.design_gradient(), sol.get_adjoint_state()))
    for o in out[1:]:
        assert o[0] == out[0][0]
        assert np.array_equal(o[1], out[0][1]) and np.array_equal(o[2], out[0][2])


def test_filtered_design_and_its_gradient_match_oracle():
    """Density filter + Heaviside projection (Sec. 3.3) on the GPU against the
    oracle, and the chain rule of the window gradient back to the raw design."""
    case = f32_inputs(I.small_channel(150, 12, window_len=12, outlet=I.OUTLET_P, tau=0.53))
    shape = (case.nz, case.ny, case.nx)
    rng = np.random.default_rng(9)
    x_raw = np.clip(I.minmax_noise(shape, 2.0, 9) * 0.8 + 0.1 * rng.random(shape), 0, 1).astype(np.float32)
    radius, beta, eta = 3.0, 4.0, 0.5
    sol = B.Solver(case, B.LBM_FP64)
    sol.set_design_filtered(x_raw, radius, beta, eta)
    gam = sol.get_design().astype(np.float64)
    phys = O.filter_project(x_raw.astype(np.float64), shape, case.design_box, radius, beta, eta)
    assert np.abs(gam - phys).max() < 1e-6
    # window + adjoint on the projected design
    pr = O.Problem(case.replace(gamma=gam.reshape(shape)))
    p0 = _developed(pr, 30)
    sol.set_state(p0)
    sol.step_window()
    sol.adjoint_window()
    g_raw = sol.design_gradient_filtered()
    _, _, _, traj = pr.run_window(p0)
    _, dgamma, _ = pr.adjoint_window(traj)
    x0, x1, y0, y1, z0, z1 = case.design_box
    m = np.zeros(shape, bool)
    m[z0:z1, y0:y1, x0:x1] = True
    dgamma = np.where(m.reshape(-1), dgamma, 0.0)          # the library's gradient is zero off the box
    want = O.filter_project_adjoint(x_raw.astype(np.float64), dgamma, shape, case.design_box, radius, beta, eta)
    assert rel_err(g_raw, want) < 1e-10


@pytest.mark.parametrize("name", ["diss-zouhe", "d3q19-pressure"])
def test_adjoint_matches_central_differences_on_the_gpu(name):
    """Single-node protocol of Sec. 4.2.1 run entirely on the GPU (FP64 path):
    central differences of the window objective (steps 2e-3 and 1e-3 on one
    FP32 design value, Richardson-extrapolated), same window and sampling
    instants, against the adjoint gradient."""
    case = f32_inputs(ADJ_CASES[name]())
    pr = O.Problem(case)
    p0 = _developed(pr, 40)
    sol = B.Solver(case, B.LBM_FP64)
    sol.set_state(p0)
    sol.step_window()
    sol.adjoint_window()
    grad = sol.design_gradient()
    gam = case.gamma.reshape(-1).astype(np.float32)
    x0, x1, y0, y1, z0, z1 = case.design_box
    rng = np.random.default_rng(4)
    nodes = []
    while len(nodes) < 4:
        x, y, z = rng.integers(x0, x1), rng.integers(y0, y1), rng.integers(z0, z1)
        i = int(x + case.nx * (y + case.ny * z))
        if 2e-3 < gam[i] < 1 - 2e-3 and abs(grad[i]) > 1e-3 * np.abs(grad).max():
            nodes.append(i)
    def central(i, step):
        js, vals = [], []
        for sgn in (1, -1):
            g2 = gam.copy()
            g2[i] += np.float32(sgn * step)
            vals.append(float(g2[i]))                 # the FP32 value actually set
            sol.set_design(g2)
            sol.set_state(p0)
            js.append(sol.step_window()[0])
        h = 0.5 * (vals[0] - vals[1])
        return (js[0] - js[1]) / (2 * h), h

    for i in nodes:
        # Richardson extrapolation of two central differences removes the h^2 term
        (d1, h1), (d2, h2) = central(i, 2e-3), central(i, 1e-3)
        fd = (h1 * h1 * d2 - h2 * h2 * d1) / (h1 * h1 - h2 * h2)
        assert abs(fd - grad[i]) <= 1e-6 * abs(grad[i]), (i, fd, grad[i])


@pytest.mark.parametrize("fmt", [I.CKPT_NATIVE, I.CKPT_BF16])
def test_pipelined_adjoint_matches_serial(fmt):
    """Recomputing segment s-1 while the adjoint sweeps segment s (two segment
    buffers, two streams) gives bitwise the serial results, with and without
    graph replay."""
    case = f32_inputs(I.small_channel(150, 12, window_len=24, ckpt_every=4, ckpt_format=fmt,
                                      outlet=I.OUTLET_P, tau=0.53))
    pr = O.Problem(case)
    p0 = _developed(pr, 20)
    out = []
    for pipeline, graphs in ((0, True), (1, True), (1, False)):
        sol = B.Solver(case, B.LBM_FP32, pipeline=pipeline)
        sol.set_graphs(graphs)
        sol.set_state(p0)
        for _ in range(2):
            sol.step_window()
            sol.adjoint_window()
        out.append((sol.design_gradient(), sol.get_adjoint_state()))
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0]) and np.array_equal(o[1], out[0][1])


def test_batch_of_replicas_matches_single_runs():
    """A D2Q9 batch (independent 2D problems as z-slices, one launch per step)
    gives each slice's window mean and gradient as a run of that problem alone
    would (FP64), and the batch matches the oracle."""
    cases = [f32_inputs(I.small_channel(140, 11, window_len=10, seed=s, outlet=I.OUTLET_P, tau=0.53,
                                        u_in=0.04 + 0.005 * s, obj_kind=k))
             for s, k in ((1, I.OBJ_DISSIPATION), (2, I.OBJ_DISSIPATION), (3, I.OBJ_DISSIPATION))]
    batch = I.stack_cases(cases)
    p0s = [_developed(O.Problem(c), 20) for c in cases]
    sol = B.Solver(batch, B.LBM_FP64)
    sol.set_state(np.concatenate(p0s, axis=1))
    Jtot, _ = sol.step_window()
    Js, _ = sol.window_objectives()
    sol.adjoint_window()
    gb = sol.design_gradient().reshape(len(cases), -1)
    assert abs(Js.sum() - Jtot) <= 1e-12 * abs(Jtot)
    for s, (c, p0) in enumerate(zip(cases, p0s)):
        one = B.Solver(c, B.LBM_FP64)
        one.set_state(p0)
        J1, _ = one.step_window()
        one.adjoint_window()
        g1 = one.design_gradient()
        assert abs(Js[s] - J1) <= 1e-12 * abs(J1)
        assert rel_err(gb[s], g1) < 1e-12
    pr = O.Problem(batch)
    _, Jw, _, traj = pr.run_window(np.concatenate(p0s, axis=1))
    _, gw, _ = pr.adjoint_window(traj)
    assert abs(Jtot - Jw) <= 1e-12 * abs(Jw)
    x0, x1, y0, y1, z0, z1 = batch.design_box
    m = np.zeros((batch.nz, batch.ny, batch.nx), bool)
    m[z0:z1, y0:y1, x0:x1] = True
    assert rel_err(gb.reshape(-1)[m.reshape(-1)], gw[m.reshape(-1)]) < 1e-11


def test_finite_difference_protocol_as_one_batch():
    """The single-node protocol of Sec. 4.2.1 as one batched run: slice 0 is
    the base design, the others carry +-h perturbations of selected nodes; the
    per-slice window means give central differences (Richardson over two
    steps) that match the base slice's adjoint gradient."""
    base = f32_inputs(I.small_channel(140, 11, window_len=10, outlet=I.OUTLET_P, tau=0.53))
    p0 = _developed(O.Problem(base), 30)
    gam = base.gamma.astype(np.float32)
    nodes = [(5, 30), (6, 70), (4, 100)]
    steps = (2e-3, 1e-3)
    cases, vals = [base], []
    for (y, x) in nodes:
        for h in steps:
            for sgn in (1, -1):
                g2 = gam.copy()
                g2[0, y, x] += np.float32(sgn * h)
                vals.append(float(g2[0, y, x]))
                cases.append(base.replace(gamma=g2.astype(np.float64)))
    batch = I.stack_cases(cases)
    sol = B.Solver(batch, B.LBM_FP64)
    sol.set_state(np.concatenate([p0] * len(cases), axis=1))
    sol.step_window()
    Js, _ = sol.window_objectives()
    sol.adjoint_window()
    grad0 = sol.design_gradient().reshape(len(cases), base.ny, base.nx)[0]
    k = 1
    for n, (y, x) in enumerate(nodes):
        d = []
        for h in steps:
            vp, vm = vals[k - 1], vals[k]
            d.append(((Js[k] - Js[k + 1]) / (vp - vm), 0.5 * (vp - vm)))
            k += 2
        (d1, h1), (d2, h2) = d
        fd = (h1 * h1 * d2 - h2 * h2 * d1) / (h1 * h1 - h2 * h2)
        assert abs(fd - grad0[y, x]) <= 1e-6 * abs(grad0[y, x]), (y, x, fd, grad0[y, x])


def test_outer_loop_in_the_library_matches_window_by_window():
    """lbm_run_until_converged (Alg. 1's outer loop) gives the windows, means and
    ratio of calling lbm_step_window one window at a time, returns
    LBM_NOT_CONVERGED at its cap, and leaves a recorded window the adjoint can
    follow."""
    case = f32_inputs(I.small_channel(140, 12, window_len=15, outlet=I.OUTLET_P, tau=0.53))
    ref = B.Solver(case, B.LBM_FP64)
    rec = ref.run_until_converged(max_windows=40)
    sol = B.Solver(case, B.LBM_FP64)
    w, J, M, ratio, conv = sol.run_windows(40)
    assert w == len(rec) and J == rec[-1]["J"] and M == rec[-1]["M"]
    assert conv == rec[-1]["converged"] and ratio == rec[-1]["ratio"]
    capped = B.Solver(case, B.LBM_FP64)
    w1, J1, _, r1, conv1 = capped.run_windows(1)
    assert w1 == 1 and not conv1 and r1 == float("inf") and J1 == rec[0]["J"]
    assert "did not hold" in B.last_error()
    capped.adjoint_window()
    assert np.abs(capped.design_gradient()).max() > 0
