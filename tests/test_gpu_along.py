"""lbm_step_window_along: one window of a context along another context's
trajectory (each checkpoint segment restarts from the reference's
checkpoint, decoded and converted).

Exact identities pin it: in the same precision and arithmetic, a window along
a native-checkpoint reference reproduces that reference's window sums,
adjoint and gradient bitwise; along a BF16-checkpoint reference it reproduces
the reference's gradient bitwise (both adjoints recompute every segment from
the same decoded start).  Across precisions it is the same-trajectory FP64
comparison of the FP32 adjoint.
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


def _case(**kw):
    return f32_inputs(I.small_channel(150, 12, window_len=24, ckpt_every=4, outlet=I.OUTLET_P,
                                      profile="parabolic", tau=0.53, cs_smag=0.12,
                                      obj_kind=I.OBJ_DISSIPATION, **kw))


def _p0(case):
    pr = O.Problem(case)
    return oracle_advance(pr, initial_flow(pr), 30)


def _reference(case, prec, p0):
    ref = B.Solver(case, prec)
    ref.set_state(p0)
    rec = ref.step_window()
    return ref, rec


@pytest.mark.parametrize("graphs", [True, False])
def test_along_a_native_reference_reproduces_it_bitwise(graphs):
    case = _case()
    p0 = _p0(case)
    ref, rec = _reference(case, B.LBM_FP32, p0)
    ctx = B.Solver(case, B.LBM_FP32)
    ctx.set_graphs(graphs)
    assert ctx.step_window_along(ref) == rec
    assert ctx.adjoint_window() == ref.adjoint_window()
    assert np.array_equal(ctx.design_gradient(), ref.design_gradient())
    assert np.array_equal(ctx.get_adjoint_state(), ref.get_adjoint_state())
    assert np.array_equal(ctx.get_state(), ref.get_state())


def test_along_a_bf16_reference_reproduces_its_gradient_bitwise():
    case = _case()
    p0 = _p0(case)
    ref, _ = _reference(case.replace(ckpt_format=I.CKPT_BF16), B.LBM_FP32, p0)
    ctx = B.Solver(case, B.LBM_FP32)
    ctx.step_window_along(ref)
    ctx.adjoint_window()
    ref.adjoint_window()
    assert np.array_equal(ctx.design_gradient(), ref.design_gradient())
    assert np.array_equal(ctx.get_adjoint_state(), ref.get_adjoint_state())


def test_fp64_along_fp32_is_the_same_trajectory_comparison():
    case = _case()
    p0 = _p0(case)
    ref, (J32, _) = _reference(case, B.LBM_FP32, p0)
    ref.adjoint_window()
    g32 = ref.design_gradient()
    ctx = B.Solver(case, B.LBM_FP64)
    J64, _ = ctx.step_window_along(ref)
    ctx.adjoint_window()
    g64 = ctx.design_gradient()
    assert J32 == pytest.approx(J64, rel=1e-5)
    assert g32 @ g64 / (np.linalg.norm(g32) * np.linalg.norm(g64)) > 0.99999
    assert np.linalg.norm(g32 - g64) <= 1e-4 * np.linalg.norm(g64)


def test_along_rejects_mismatches():
    case = _case()
    ref = B.Solver(case, B.LBM_FP32)
    ctx = B.Solver(case, B.LBM_FP32)
    with pytest.raises(B.LbmError) as e:          # no completed window yet
        ctx.step_window_along(ref)
    assert e.value.status == B.LBM_ERR_STATE
    ref.set_state(_p0(case))
    ref.step_window()
    other = B.Solver(case.replace(ckpt_every=6), B.LBM_FP32)
    with pytest.raises(B.LbmError) as e:
        other.step_window_along(ref)
    assert e.value.status == B.LBM_ERR_ARG
    mom = B.Solver(case.replace(ckpt_format=I.CKPT_MOMENT), B.LBM_FP32)
    with pytest.raises(B.LbmError) as e:
        mom.step_window_along(ref)
    assert e.value.status == B.LBM_ERR_ARG
    with pytest.raises(B.LbmError):
        ctx.step_window_along(ctx)
