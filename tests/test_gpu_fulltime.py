"""Full-time adjoint runs (Sec. 4.2.3) through the C ABI.

A full-time run is one window of T steps from the initial field whose
samples start at step T - |W| (lbm_set_sample_start): the objective is the
mean over the final |W| steps, and lbm_adjoint_window traces the adjoint back
to the initial time through every checkpoint segment.  Checked here:

* J, the monitor, the design gradient and the start-field adjoint against the
  FP64 oracle's full-time run (tolerances of test_gpu_parity.py: 1e-12 for the
  FP64 build; cosine 0.9999 and 1e-3 norm-wise for FP32);
* J and the final state equal, bit for bit, a plain window after the same
  unsampled spin-up (same samples, same block sums, same reduction);
* the pipelined launch path;
* argument and state errors of lbm_set_sample_start.
"""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2608_19617_b300 import binding as B
from paper_2608_19617_b300 import inputs as I

from _util import cosine, f32_inputs, initial_flow, oracle_advance, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2608_19617_b300 import build
    build.build()
    B.lib()


# (case, first sampled step)
CASES = {
    "diss-zouhe-every2": (lambda: I.small_channel(150, 12, obj_kind=I.OBJ_DISSIPATION, window_len=16, ckpt_every=4,
                                                  sample_every=2, outlet=I.OUTLET_P, profile="parabolic",
                                                  tau=0.53, cs_smag=0.12), 8),
    "veldev-zg-odd-start": (lambda: I.small_channel(140, 11, obj_kind=I.OBJ_VELOCITY_DEV, window_len=15,
                                                    ckpt_every=5, outlet=I.OUTLET_ZG, tau=0.52), 7),
    "drag-periodic": (lambda: I.small_channel(129, 9, obj_kind=I.OBJ_DRAG, window_len=12, ckpt_every=3,
                                              periodic_x=True, g_max=0.9), 6),
    "d3q19-pressure": (lambda: I.small_duct3d(130, 6, 6, window_len=10, ckpt_every=5, tau=0.53), 4),
}


def _full_time(name):
    make, first = CASES[name]
    return f32_inputs(make()).replace(sample_from=first)


def _design_mask(case):
    m = np.zeros((case.nz, case.ny, case.nx), bool)
    x0, x1, y0, y1, z0, z1 = case.design_box
    m[z0:z1, y0:y1, x0:x1] = True
    return m.reshape(-1)


def _gpu_run(case, precision, p0, **kw):
    sol = B.Solver(case, precision, **kw)
    sol.set_state(p0)
    J, M = sol.step_window()
    Jeff = sol.adjoint_window()
    out = dict(J=J, M=M, Jeff=Jeff, grad=sol.design_gradient(), a0=sol.get_adjoint_state(), state=sol.get_state())
    sol.close()
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_full_time_run_fp64_matches_oracle(name):
    case = _full_time(name)
    pr = O.Problem(case)
    p0 = initial_flow(pr)
    _, Jw, Mw, traj = pr.run_window(p0)
    _, grad_w, a0_w = pr.adjoint_window(traj)
    got = _gpu_run(case, B.LBM_FP64, p0)
    assert abs(got["J"] - Jw) <= 1e-12 * abs(Jw)
    assert abs(got["M"] - Mw) <= 1e-12 * abs(Mw) + 1e-300
    assert got["Jeff"] == got["J"]
    m = _design_mask(case)
    assert rel_err(got["grad"][m], grad_w[m]) < 1e-11
    assert np.all(got["grad"][~m] == 0)
    assert rel_err(got["a0"], a0_w) < 1e-11


@pytest.mark.parametrize("name", list(CASES))
def test_full_time_run_fp32_matches_oracle(name):
    case = _full_time(name)
    pr = O.Problem(case)
    p0 = initial_flow(pr)
    _, Jw, _, traj = pr.run_window(p0)
    _, grad_w, a0_w = pr.adjoint_window(traj)
    got = _gpu_run(case, B.LBM_FP32, p0)
    assert abs(got["J"] - Jw) <= 1e-4 * abs(Jw)
    m = _design_mask(case)
    assert cosine(got["grad"][m], grad_w[m]) > 0.9999
    assert rel_err(got["grad"][m], grad_w[m]) < 1e-3
    assert cosine(got["a0"], a0_w) > 0.9999


@pytest.mark.parametrize("graphs", [True, False])
@pytest.mark.parametrize("name", ["diss-zouhe-every2", "d3q19-pressure"])
def test_full_time_objective_is_the_final_window_bitwise(name, graphs):
    """J, monitor and final state of the full-time run equal those of a plain
    window of T - s0 steps after s0 unsampled steps, bit for bit."""
    case = _full_time(name)
    T, s0 = case.window_len, case.sample_from
    p0 = initial_flow(O.Problem(case))
    full = B.Solver(case, B.LBM_FP32)
    full.set_graphs(graphs)
    full.set_state(p0)
    Jf, Mf = full.step_window()
    sf = full.get_state()
    full.close()
    win_case = case.replace(window_len=T - s0, ckpt_every=T - s0, sample_from=0)
    win = B.Solver(win_case, B.LBM_FP32)
    win.set_graphs(graphs)
    win.set_state(p0)
    win.advance(s0)
    Jw, Mw = win.step_window()
    sw = win.get_state()
    win.close()
    assert Jf == Jw and Mf == Mw
    assert np.array_equal(sf, sw)


def test_full_time_on_the_pipelined_path():
    """The pipelined sweep (two segment buffers) against the serial sweep of
    the same full-time run, bit for bit."""
    case = _full_time("diss-zouhe-every2")
    p0 = oracle_advance(O.Problem(case), initial_flow(O.Problem(case)), 5)
    ref = _gpu_run(case, B.LBM_FP32, p0, pipeline=0)
    pipe = _gpu_run(case, B.LBM_FP32, p0, pipeline=1)
    assert pipe["J"] == ref["J"]
    assert np.array_equal(pipe["grad"], ref["grad"]) and np.array_equal(pipe["a0"], ref["a0"])


def test_sample_start_arguments_and_state():
    case = f32_inputs(I.small_channel(64, 10, window_len=12, ckpt_every=4, sample_every=3))
    sol = B.Solver(case, B.LBM_FP32)
    for bad in (-1, 12, 13, 4, 10):      # outside [0, 12) or 12 - first not a multiple of 3
        with pytest.raises(B.LbmError) as e:
            sol.set_sample_start(bad)
        assert e.value.status == B.LBM_ERR_ARG
    sol.step_window()
    sol.set_sample_start(3)              # invalidates the recorded window
    with pytest.raises(B.LbmError) as e:
        sol.adjoint_window()
    assert e.value.status == B.LBM_ERR_STATE
    sol.step_window()
    sol.adjoint_window()
    sol.set_sample_start(0)
    sol.close()
