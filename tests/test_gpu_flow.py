"""Persistent segment launches (lbm_set_flow) against the per-step kernels.

A persistent launch runs the K steps of a checkpoint segment in one
cooperative kernel whose blocks own bands of nodes and wait only for the bands
they exchange data with.  Every node is computed by the same node function as
in the per-step kernels, compiled in another context (the compiler may fuse
multiply-adds differently), so states, adjoint fields and gradients agree to
a few units in the last place of the working precision; window sums are added
in another grouping.  A missed dependency would instead mix in a neighbour's
value from the previous step, an error of order |p^n - p^(n-1)| ~ 1e-4 here.
The per-step kernels are themselves checked against the oracle in
test_gpu_parity.py.
"""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2608_19617_b300 import binding as B
from paper_2608_19617_b300 import inputs as I

from _util import f32_inputs, initial_flow, oracle_advance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2608_19617_b300 import build
    build.build()
    B.lib()


CASES = {
    "d2-zouhe-fp32": (lambda: I.small_channel(150, 12, window_len=12, ckpt_every=4, outlet=I.OUTLET_P,
                                              profile="parabolic", tau=0.53, cs_smag=0.12,
                                              obj_kind=I.OBJ_DISSIPATION), B.LBM_FP32),
    "d2-zerograd-every3-fp64": (lambda: I.small_channel(140, 11, window_len=12, ckpt_every=6, outlet=I.OUTLET_ZG,
                                                        sample_every=3, tau=0.52, obj_kind=I.OBJ_VELOCITY_DEV),
                                B.LBM_FP64),
    "d2-periodic-drag-oddK-fp32": (lambda: I.small_channel(129, 9, window_len=15, ckpt_every=5, periodic_x=True,
                                                           g_max=0.9, obj_kind=I.OBJ_DRAG), B.LBM_FP32),
    "d2-pressure-K1-fp32": (lambda: I.small_channel(133, 10, window_len=6, ckpt_every=1,
                                                    obj_kind=I.OBJ_PRESSURE, tau=0.56), B.LBM_FP32),
    "d3-pressure-fp32": (lambda: I.small_duct3d(130, 6, 6, window_len=8, ckpt_every=4, tau=0.53), B.LBM_FP32),
    "d3-diss-periodicz-fp64": (lambda: I.small_duct3d(131, 6, 5, window_len=8, ckpt_every=2, periodic_z=True,
                                                      obj_kind=I.OBJ_DISSIPATION, tau=0.54), B.LBM_FP64),
}


def _start(case, steps=20):
    pr = O.Problem(case)
    return oracle_advance(pr, initial_flow(pr), steps)


def _advanced(case, steps):
    """A developed start field from the GPU path itself.  Every run under
    comparison then loads it through set_state: the FP64 round trip of
    get_state / set_state is not the identity for near-rest populations."""
    sol = B.Solver(case, B.LBM_FP32)
    sol.advance(steps)
    p0 = sol.get_state()
    sol.close()
    return p0


def _run(case, precision, flow, p0, windows=2, graphs=True, **kw):
    sol = B.Solver(case, precision, **kw)
    sol.set_graphs(graphs)
    if flow:
        sol.set_flow(True)
    sol.set_state(p0)
    rec = [sol.step_window() for _ in range(windows)]
    conv = sol.window_converged()
    Jeff = sol.adjoint_window()
    out = dict(rec=rec, conv=conv, Jeff=Jeff, grad=sol.design_gradient(), a0=sol.get_adjoint_state(),
               state=sol.get_state(), sched=sol.schedule())
    sol.close()
    return out


def _close(x, y, eps):
    """max |x - y| within 64 ulps of the largest entry (rounding, not a stale read)."""
    scale = max(float(np.abs(y).max()), 1e-300)
    assert float(np.abs(x - y).max()) <= 64 * eps * scale


def _same(a, b, rtol):
    eps = 2.0 ** -23 if rtol > 1e-9 else 2.0 ** -52
    _close(a["state"], b["state"], eps)
    _close(a["a0"], b["a0"], eps)
    _close(a["grad"], b["grad"], 16 * eps)
    for (ja, ma), (jb, mb) in zip(a["rec"], b["rec"]):
        assert ja == pytest.approx(jb, rel=rtol, abs=1e-300)
        assert ma == pytest.approx(mb, rel=rtol, abs=1e-300)
    assert a["Jeff"] == pytest.approx(b["Jeff"], rel=rtol, abs=1e-300)


@pytest.mark.parametrize("name", list(CASES))
def test_persistent_segments_match_per_step_kernels(name):
    make, prec = CASES[name]
    case = make()
    if prec == B.LBM_FP32:
        case = f32_inputs(case)
    p0 = _start(case)
    ref = _run(case, prec, False, p0)
    rtol = 2e-6 if prec == B.LBM_FP32 else 1e-12
    for graphs in (True, False):
        got = _run(case, prec, True, p0, graphs=graphs)
        assert got["sched"]["flow"] == 1 and got["sched"]["flow_bands"] >= 2
        _same(got, ref, rtol)


@pytest.mark.parametrize("fmt", [I.CKPT_FP16, I.CKPT_BF16])
def test_persistent_segments_with_sixteen_bit_checkpoints(fmt):
    case = f32_inputs(I.small_channel(150, 12, window_len=24, ckpt_every=4, ckpt_format=fmt,
                                      outlet=I.OUTLET_P, tau=0.53))
    p0 = _start(case)
    ref = _run(case, B.LBM_FP32, False, p0)
    got = _run(case, B.LBM_FP32, True, p0)
    _same(got, ref, 2e-6)


def test_persistent_segments_ignore_the_pipeline_flag():
    """With pipeline=1 the persistent sweep runs serially (one cooperative
    kernel at a time) and still matches the pipelined per-step sweep."""
    case = f32_inputs(I.small_channel(150, 12, window_len=24, ckpt_every=4, outlet=I.OUTLET_P, tau=0.53))
    p0 = _start(case)
    ref = _run(case, B.LBM_FP32, False, p0, pipeline=1)
    got = _run(case, B.LBM_FP32, True, p0, pipeline=1)
    _same(got, ref, 2e-6)


@pytest.mark.parametrize("name", ["wake1024x256", "ubend256x128x64"])
def test_persistent_segments_at_full_size(name):
    """Full-size lattices (hundreds of bands), a short window: states and
    gradient against the per-step kernels."""
    case = I.WORKLOADS[name]()
    case = case.replace(window_len=2 * case.ckpt_every if case.lattice == 9 else 20,
                        ckpt_every=case.ckpt_every if case.lattice == 9 else 10)
    p0 = _advanced(case, 300)
    out = []
    for flow in (False, True):
        sol = B.Solver(case, B.LBM_FP32)
        if flow:
            sol.set_flow(True)
        sol.set_state(p0)
        rec = sol.step_window()
        sol.adjoint_window()
        out.append((rec, sol.get_state(), sol.design_gradient(), sol.schedule()))
        sol.close()
    (r0, s0, g0, _), (r1, s1, g1, sc) = out
    assert sc["flow_bands"] >= 100
    _close(s1, s0, 2.0 ** -23)
    _close(g1, g0, 16 * 2.0 ** -23)
    assert r1[0] == pytest.approx(r0[0], rel=1e-5) and r1[1] == pytest.approx(r0[1], rel=1e-5)


def _forward_states(case, prec, p0, windows):
    out = []
    for flow in (False, True):
        sol = B.Solver(case, prec)
        if flow:
            sol.set_flow(True)
        sol.set_state(p0)
        for _ in range(windows):
            sol.step_window()
        out.append(sol.get_state())
        sol.close()
    return out


@pytest.mark.parametrize("name", ["d2-zouhe-fp32", "d2-zerograd-every3-fp64", "d3-pressure-fp32",
                                  "d3-diss-periodicz-fp64"])
def test_geometric_face_nodes_match_the_face_table_bitwise(name):
    """The per-step face kernels take a face node's position, class and
    sources from the geometry; the persistent kernels read them from the
    host-built face table.  The node arithmetic is explicitly rounded, so the
    forward states agree bit for bit (a wrong source, mask or inlet velocity
    would not)."""
    make, prec = CASES[name]
    case = make()
    if prec == B.LBM_FP32:
        case = f32_inputs(case)
    s0, s1 = _forward_states(case, prec, _start(case), 2)
    assert np.array_equal(s0, s1)


def test_geometric_face_nodes_match_the_face_table_on_the_ubend():
    """Full-size U-bend (velocity inlet and zero-gradient outlet on the x = 0
    face, walls elsewhere): geometric and table face nodes, bit for bit."""
    case = I.WORKLOADS["ubend256x128x64"]()
    case = case.replace(window_len=20, ckpt_every=10)
    s0, s1 = _forward_states(case, B.LBM_FP32, _advanced(case, 60), 1)
    assert np.array_equal(s0, s1)


def test_persistent_segments_are_rejected_for_batches():
    case = I.stack_cases([I.small_channel(64, 10, window_len=4, ckpt_every=2) for _ in range(2)])
    sol = B.Solver(case, B.LBM_FP32)
    assert sol.schedule()["flow_bands"] == 0
    with pytest.raises(B.LbmError) as e:
        sol.set_flow(True)
    assert e.value.status == B.LBM_ERR_ARG
    sol.close()


def test_a_wait_that_runs_out_fails_the_window_and_the_context_recovers():
    """Band 0 never publishes its progress: its neighbours' bounded waits run
    out (0.2 s), every block leaves, the window reports LBM_ERR_CUDA, and
    the same context then runs a correct window and sweep."""
    case = f32_inputs(I.small_channel(150, 12, window_len=12, ckpt_every=4, outlet=I.OUTLET_P, tau=0.53))
    p0 = _start(case)
    ref = _run(case, B.LBM_FP32, False, p0, windows=1)
    sol = B.Solver(case, B.LBM_FP32)
    sol.set_flow(True)
    sol.set_flow_test_hook(0.2, 0)
    sol.set_state(p0)
    with pytest.raises(B.LbmError) as e:
        sol.step_window()
    assert e.value.status == B.LBM_ERR_CUDA and "timed out" in str(e.value)
    sol.set_flow_test_hook(4.0, -1)
    sol.set_state(p0)
    rec = sol.step_window()
    sol.adjoint_window()
    assert rec[0] == pytest.approx(ref["rec"][0][0], rel=2e-6)
    _close(sol.get_state(), ref["state"], 2.0 ** -23)
    _close(sol.design_gradient(), ref["grad"], 16 * 2.0 ** -23)
    sol.close()
