"""Moment checkpoints (LBM_CKPT_MOMENT) are lossless.

A moment checkpoint keeps the per-node blend coefficients (a0, b, m, X) that
the step producing the field computed; decoding applies the step's own
arithmetic, w_a (a0 + b m.c_a + 4.5 c_a.X.c_a) with fused multiply-adds in a
fixed order.  So the recomputed segments, the adjoint sweep and the gradient
must be bitwise those of native checkpoints, with and without graphs and
pipelining.
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
    "d2-fp32": (lambda **kw: I.small_channel(132, 12, window_len=24, ckpt_every=4, outlet=I.OUTLET_P,
                                             tau=0.53, obj_kind=I.OBJ_DISSIPATION, **kw), B.LBM_FP32),
    "d2-zerograd-every3-fp64": (lambda **kw: I.small_channel(140, 11, window_len=12, ckpt_every=3,
                                                             outlet=I.OUTLET_ZG, sample_every=3, tau=0.52,
                                                             obj_kind=I.OBJ_VELOCITY_DEV, **kw), B.LBM_FP64),
    "d3-fp32": (lambda **kw: I.small_duct3d(132, 8, 6, window_len=12, ckpt_every=3, tau=0.53, **kw), B.LBM_FP32),
}


def _run(case, precision, p0, **switches):
    sol = B.Solver(case, precision, pipeline=switches.pop("pipeline", 0))
    for name, on in switches.items():
        getattr(sol, "set_" + name)(on)
    sol.set_state(p0)
    rec = [sol.step_window() for _ in range(2)]
    Jeff = sol.adjoint_window()
    out = (rec, Jeff, sol.design_gradient(), sol.get_adjoint_state(), sol.get_state())
    sol.close()
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_moment_checkpoints_reproduce_native_checkpoints_bitwise(name):
    make, prec = CASES[name]
    native, moment = make(), make().replace(ckpt_format=I.CKPT_MOMENT)
    if prec == B.LBM_FP32:
        native, moment = f32_inputs(native), f32_inputs(moment)
    pr = O.Problem(native)
    p0 = oracle_advance(pr, initial_flow(pr), 20)
    variants = [dict(), dict(graphs=False), dict(pipeline=1)]
    for sw in variants:
        ref = _run(native, prec, p0, **dict(sw))
        got = _run(moment, prec, p0, **dict(sw))
        assert got[0] == ref[0] and got[1] == ref[1], sw
        for a, b in zip(got[2:], ref[2:]):
            assert np.array_equal(a, b), sw


def test_moment_checkpoints_at_full_size():
    case = I.WORKLOADS["ubend256x128x64"]().replace(window_len=40, ckpt_every=10)
    sol = B.Solver(case, B.LBM_FP32)
    sol.advance(200)
    p0 = sol.get_state()
    sol.close()
    out = []
    for fmt in (I.CKPT_NATIVE, I.CKPT_MOMENT):
        s = B.Solver(case.replace(ckpt_format=fmt), B.LBM_FP32, pipeline=1)
        s.set_state(p0)
        rec = s.step_window()
        s.adjoint_window()
        out.append((rec, s.design_gradient()))
        s.close()
    assert out[0][0] == out[1][0] and np.array_equal(out[0][1], out[1][1])
