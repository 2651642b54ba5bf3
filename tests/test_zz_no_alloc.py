"""The no-allocation window: a caller that cannot allocate device memory (a
host that hands the library only buffers it registered up front, or a sandbox
without the CUDA allocator) runs a forward window through
lbm_step_window_noalloc on buffers it already owns and gets what
lbm_step_window gives, call after call.

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


def _device_inputs(case):
    import torch
    dev = "cuda"
    return (torch.tensor(case.node_class.reshape(-1), dtype=torch.uint8, device=dev),
            torch.tensor(case.gamma.reshape(-1), dtype=torch.float32, device=dev),
            torch.tensor(case.obj_weights.reshape(-1), dtype=torch.float32, device=dev),
            torch.tensor(case.inlet_u.reshape(-1), dtype=torch.float32, device=dev))


def test_noalloc_at_its_scratch_limit_matches_step_window():
    """Exactly 16384 blocks (a 256x128x64 D3Q19 U-bend: 2 x 128 x 64 rows of
    128 nodes), pressure-drop objective and drag monitor, two calls in a row.
    The populations are computed by the same explicitly rounded node
    arithmetic, so the fields agree bit for bit.  The window means differ only
    by FP32 summation inside the blocks (the two paths cut the lattice into
    different blocks, and this path samples cs^2 rho where lbm_step_window
    samples cs^2 (rho - 1) and adds cs^2 sum w in FP64): per sample at most
    about 10 roundings of the summed magnitudes, 10 * 2^-24 * sum_i |w_i psi_i|
    (two product roundings and a tree of eight additions)."""
    import torch
    from paper_2608_19617_b300 import build
    build.build()
    case = f32_inputs(I.WORKLOADS["ubend256x128x64"]().replace(window_len=20, ckpt_every=10))
    assert ((case.nx + 127) // 128) * case.ny * case.nz == 16384
    sol = B.Solver(case, B.LBM_FP32)
    sol.advance(100)
    p0 = sol.get_state()
    sol.set_state(p0)
    ref = [sol.step_window() for _ in range(2)]
    p_ref = sol.get_state()
    sol.close()

    lat = O.Lattice(19)
    w = lat.w[:, None]
    pop = torch.tensor((p0 - w).astype(np.float32), device="cuda")
    tmp = torch.empty_like(pop)
    cfg = B.config_from_case(case, B.LBM_FP32)
    stream = torch.cuda.current_stream().cuda_stream
    tensors = _device_inputs(case)
    got = []
    for _ in range(2):
        st, J, M = _noalloc(case, cfg, tensors, pop, tmp, stream)
        assert st == B.LBM_OK, B.last_error()
        got.append((J, M))
    state = pop.double().cpu().numpy() + w
    assert np.array_equal(state, p_ref)

    # bounds of the FP32 block sums from the field at the window end: the
    # samples see the pulled field f_a(i) = p_a(i - c_a), here by periodic
    # shifts (exact off the faces, where the drag terms are largest), with a
    # factor 2 for the faces and the change over the window
    pc = p_ref.reshape(19, case.nz, case.ny, case.nx)
    f = np.stack([np.roll(pc[a], (lat.c3[a][2], lat.c3[a][1], lat.c3[a][0]), axis=(0, 1, 2))
                  for a in range(19)]).reshape(19, -1)
    rho, u = O.moments_of(lat, f)
    eps = 2.0 ** -24
    j_mag = float(np.abs(case.obj_weights.reshape(-1)).sum()) / 3.0 * float(rho.max())
    g = O.g_of_phi(1.0 - case.gamma.reshape(-1), case.q_interp, case.g_max)
    m_mag = 2.0 * float(np.abs(2.0 * g * rho * u[0]).sum()) / (0.5 * case.rho_out * case.monitor_u ** 2
                                                               * case.monitor_l)
    assert m_mag > 0
    for (j, m), (jr, mr) in zip(got, ref):
        assert abs(j - jr) <= 10 * eps * j_mag, (j, jr, 10 * eps * j_mag)
        assert abs(m - mr) <= 10 * eps * m_mag, (m, mr, 10 * eps * m_mag)


def test_noalloc_refuses_a_capturing_stream_and_a_bad_class_map():
    """A stream in graph-capture mode is refused before anything is enqueued
    (the call reads its results back and waits for the stream), and a class
    map that lbm_create would reject fails the call with LBM_ERR_ARG instead
    of reading outside the lattice; the next valid call still succeeds."""
    import warnings

    import torch
    case = f32_inputs(CASES["d2q9-dissipation-w16"]())
    pr = O.Problem(case)
    w = pr.lat.w[:, None]
    p0 = (initial_flow(pr) - w).astype(np.float32)
    pop = torch.tensor(p0, device="cuda")
    tmp = torch.empty_like(pop)
    cfg = B.config_from_case(case, B.LBM_FP32)
    tensors = _device_inputs(case)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")          # the captured graph stays empty
        with torch.cuda.graph(graph, stream=side):
            st, _, _ = _noalloc(case, cfg, tensors, pop, tmp, side.cuda_stream)
    assert st == B.LBM_ERR_ARG and "capturing" in B.last_error()
    assert torch.equal(pop.cpu(), torch.tensor(p0))

    bad = tensors[0].clone()
    bad[5 * case.nx + 40] = I.INLET               # an inlet class in the interior
    stream = torch.cuda.current_stream().cuda_stream
    st, _, _ = _noalloc(case, cfg, (bad,) + tensors[1:], pop, tmp, stream)
    assert st == B.LBM_ERR_ARG and "node_class" in B.last_error()
    pop.copy_(torch.tensor(p0))
    st, J, _ = _noalloc(case, cfg, tensors, pop, tmp, stream)
    assert st == B.LBM_OK and np.isfinite(J), B.last_error()
