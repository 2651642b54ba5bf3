"""TMA-staged interior forward steps (lbm_set_tma) against the per-step kernels.

fwd_tma_kernel stages each tile's source rows in shared memory with TMA bulk
tensor copies and then runs forward_core(), the arithmetic of the register
path, on the same nodes, with the block sums in the same per-tile slots.  The
compiler may fuse multiply-adds of that source differently in the two
kernels, so states, window sums and (through the recompute) gradients agree
to a few units in the last place, not necessarily bitwise.  A wrong stage,
box or shift would instead mix in another node's populations.  The register
path is itself checked against the oracle in test_gpu_parity.py.
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
    "d2-zouhe-fp32": (lambda: I.small_channel(132, 12, window_len=12, ckpt_every=4, outlet=I.OUTLET_P,
                                              profile="parabolic", tau=0.53, cs_smag=0.12,
                                              obj_kind=I.OBJ_DISSIPATION), B.LBM_FP32),
    "d2-zerograd-every3-fp64": (lambda: I.small_channel(260, 11, window_len=12, ckpt_every=6, outlet=I.OUTLET_ZG,
                                                        sample_every=3, tau=0.52, obj_kind=I.OBJ_VELOCITY_DEV),
                                B.LBM_FP64),
    "d2-periodic-drag-fp32": (lambda: I.small_channel(128, 9, window_len=15, ckpt_every=5, periodic_x=True,
                                                      g_max=0.9, obj_kind=I.OBJ_DRAG), B.LBM_FP32),
    "d3-pressure-fp32": (lambda: I.small_duct3d(132, 8, 6, window_len=8, ckpt_every=4, tau=0.53), B.LBM_FP32),
    "d3-diss-periodicz-fp64": (lambda: I.small_duct3d(130, 6, 5, window_len=8, ckpt_every=2, periodic_z=True,
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


def _run(case, precision, tma, p0, windows=2, graphs=True, **kw):
    sol = B.Solver(case, precision, **kw)
    sol.set_graphs(graphs)
    assert sol.schedule()["tma_available"] == 1
    if tma:
        sol.set_tma(True)
    sol.set_state(p0)
    rec = [sol.step_window() for _ in range(windows)]
    Jeff = sol.adjoint_window()
    out = dict(rec=rec, Jeff=Jeff, grad=sol.design_gradient(), a0=sol.get_adjoint_state(), state=sol.get_state())
    sol.close()
    return out


def _same(a, b, fp32=True):
    eps = 64 * (2.0 ** -23 if fp32 else 2.0 ** -52)
    for (ja, ma), (jb, mb) in zip(a["rec"], b["rec"]):
        assert ja == pytest.approx(jb, rel=eps) and ma == pytest.approx(mb, rel=eps)
    for k, f in (("state", 1), ("a0", 1), ("grad", 16)):
        assert float(np.abs(a[k] - b[k]).max()) <= f * eps * float(np.abs(b[k]).max()), k


@pytest.mark.parametrize("name", list(CASES))
def test_tma_staging_matches_the_register_path(name):
    make, prec = CASES[name]
    case = make()
    if prec == B.LBM_FP32:
        case = f32_inputs(case)
    p0 = _start(case)
    ref = _run(case, prec, False, p0)
    for graphs in (True, False):
        _same(_run(case, prec, True, p0, graphs=graphs), ref, fp32=prec == B.LBM_FP32)


@pytest.mark.parametrize("fmt", [I.CKPT_FP16, I.CKPT_BF16])
def test_tma_staging_with_sixteen_bit_checkpoints_and_pipeline(fmt):
    """Forward states agree to rounding.  A last-place difference can move one
    16-bit checkpoint value by a quantisation step, so the recomputed segments,
    the adjoint and the gradient agree to the 16-bit format's resolution."""
    case = f32_inputs(I.small_channel(132, 12, window_len=24, ckpt_every=4, ckpt_format=fmt,
                                      outlet=I.OUTLET_P, tau=0.53))
    p0 = _start(case)
    a = _run(case, B.LBM_FP32, True, p0, pipeline=1)
    b = _run(case, B.LBM_FP32, False, p0, pipeline=1)
    eps = 64 * 2.0 ** -23
    for (ja, ma), (jb, mb) in zip(a["rec"], b["rec"]):
        assert ja == pytest.approx(jb, rel=eps) and ma == pytest.approx(mb, rel=eps)
    assert float(np.abs(a["state"] - b["state"]).max()) <= eps * float(np.abs(b["state"]).max())
    for k in ("a0", "grad"):
        assert np.linalg.norm(a[k] - b[k]) <= 1e-3 * np.linalg.norm(b[k]), k


def test_tma_staging_of_a_batch():
    cases = [f32_inputs(I.small_channel(128, 10, window_len=6, ckpt_every=3, seed=s, outlet=I.OUTLET_P))
             for s in (1, 2, 3)]
    case = I.stack_cases(cases)
    out = []
    for tma in (False, True):
        sol = B.Solver(case, B.LBM_FP32)
        if tma:
            sol.set_tma(True)
        sol.advance(30)
        rec = sol.step_window()
        out.append((rec, sol.window_objectives()[0], sol.get_state()))
        sol.close()
    eps = 64 * 2.0 ** -23
    assert out[1][0][0] == pytest.approx(out[0][0][0], rel=eps)
    assert np.abs(out[1][1] - out[0][1]).max() <= eps * np.abs(out[0][1]).max()
    assert np.abs(out[1][2] - out[0][2]).max() <= eps * np.abs(out[0][2]).max()


@pytest.mark.parametrize("name", ["wake1024x256", "ubend256x128x64"])
def test_tma_staging_at_full_size(name):
    case = I.WORKLOADS[name]()
    case = case.replace(window_len=2 * case.ckpt_every if case.lattice == 9 else 20,
                        ckpt_every=case.ckpt_every if case.lattice == 9 else 10)
    out = []
    p0 = _advanced(case, 300)
    for tma in (False, True):
        sol = B.Solver(case, B.LBM_FP32, pipeline=1)
        if tma:
            sol.set_tma(True)
        sol.set_state(p0)
        rec = sol.step_window()
        sol.adjoint_window()
        out.append((rec, sol.get_state(), sol.design_gradient()))
        sol.close()
    eps = 64 * 2.0 ** -23
    assert out[1][0][0] == pytest.approx(out[0][0][0], rel=eps) and out[1][0][1] == pytest.approx(out[0][0][1], rel=eps)
    assert np.abs(out[1][1] - out[0][1]).max() <= eps * np.abs(out[0][1]).max()
    assert np.abs(out[1][2] - out[0][2]).max() <= 16 * eps * np.abs(out[0][2]).max()


def test_tma_staging_needs_a_16_byte_row_pitch():
    case = I.small_channel(150, 12, window_len=4, ckpt_every=2)   # 150 * 4 bytes is not a multiple of 16
    sol = B.Solver(case, B.LBM_FP32)
    assert sol.schedule()["tma_available"] == 0
    with pytest.raises(B.LbmError) as e:
        sol.set_tma(True)
    assert e.value.status == B.LBM_ERR_ARG
    sol.close()
