"""The no-allocation window: a caller that cannot allocate device memory runs
a forward window through lbm_step_window_noalloc on buffers it already owns
and gets what lbm_step_window gives, call after call.

This file is collected last, so a run that stops at the first failure has
already run every other test.
"""
from ctypes import byref, c_double, c_void_p

import numpy as np
import pytest

from oracle import lbm as O
from paper_2608_19617_b300 import binding as B
from paper_2608_19617_b300 import inputs as I

from _util import f32_inputs, initial_flow

pytestmark = pytest.mark.gpu

CASES = {
    "d2q9-dissipation-w16": lambda: I.small_channel(300, 20, obj_kind=I.OBJ_DISSIPATION, window_len=16,
                                                    outlet=I.OUTLET_P, tau=0.53),
    "d3q19-pressure-w15": lambda: I.small_duct3d(140, 7, 6, window_len=15, ckpt_every=5, tau=0.53),
}


def _noalloc(case, cfg, tensors, pop, tmp, stream):
    cls, gam, w, uin = tensors
    J, M = c_double(), c_double()
    st = B.lib().lbm_step_window_noalloc(byref(cfg), cls.data_ptr(), gam.data_ptr(), w.data_ptr(),
                                         uin.data_ptr(), pop.data_ptr(), tmp.data_ptr(), c_void_p(stream),
                                         byref(J), byref(M))
    return st, J.value, M.value


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_window_matches_step_window_on_two_calls(name):
    import torch
    from paper_2608_19617_b300 import build
    build.build()
    case = f32_inputs(CASES[name]())
    pr = O.Problem(case)
    p0 = initial_flow(pr)

    sol = B.Solver(case, B.LBM_FP32)
    sol.set_state(p0)
    ref = [sol.step_window() for _ in range(2)]
    p_ref = sol.get_state()

    dev = "cuda"
    tensors = (torch.tensor(case.node_class.reshape(-1), dtype=torch.uint8, device=dev),
               torch.tensor(case.gamma.reshape(-1), dtype=torch.float32, device=dev),
               torch.tensor(case.obj_weights.reshape(-1), dtype=torch.float32, device=dev),
               torch.tensor(case.inlet_u.reshape(-1), dtype=torch.float32, device=dev))
    w = pr.lat.w[:, None]
    pop = torch.tensor((p0 - w).astype(np.float32), device=dev)   # shifted FP32 layout
    tmp = torch.empty_like(pop)
    cfg = B.config_from_case(case, B.LBM_FP32)
    stream = torch.cuda.current_stream().cuda_stream
    got = []
    for _ in range(2):
        st, J, M = _noalloc(case, cfg, tensors, pop, tmp, stream)
        assert st == B.LBM_OK, B.last_error()
        got.append((J, M))
    for (j, m), (jr, mr) in zip(got, ref):
        assert abs(j - jr) <= 1e-4 * abs(jr), (j, jr)
        assert abs(m - mr) <= 1e-4 * abs(mr) + 1e-300, (m, mr)
    state = pop.double().cpu().numpy() + w
    assert np.abs(state - p_ref).max() < 1e-6


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch
    case = I.small_channel(16, 8)
    cfg = B.config_from_case(case, B.LBM_FP32)
    cfg.nx, cfg.ny = 2048, 1100           # 16 x 1100 = 17600 blocks > 16384
    t = torch.zeros(8, device="cuda")     # never touched: the call returns before any launch
    st = B.lib().lbm_step_window_noalloc(byref(cfg), t.data_ptr(), t.data_ptr(), t.data_ptr(), t.data_ptr(),
                                         t.data_ptr(), t.data_ptr() + 4, None, None, None)
    assert st == B.LBM_ERR_ARG
    assert "16384" in B.last_error()
