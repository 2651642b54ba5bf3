"""The C ABI without a GPU: the library loads, exports every declared entry
point, and rejects invalid configurations on the host before any CUDA call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2608_19617_b300 import binding as B, build
from paper_2608_19617_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return B.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbmadj.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_struct_layouts_match_the_c_compiler(lib, tmp_path):
    """Offsets of every field of lbm_config / lbm_timing / lbm_schedule as gcc
    lays them out from the header equal the ctypes mirror's."""
    fields = [f for f, _ in B.LbmConfig._fields_]
    tfields = [f for f, _ in B.LbmTiming._fields_]
    sfields = [f for f, _ in B.LbmSchedule._fields_]
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbmadj.h"', "int main(void){"]
    prog.append('printf("%zu\\n", sizeof(lbm_config));')
    prog += [f'printf("%zu\\n", offsetof(lbm_config, {f}));' for f in fields]
    prog.append('printf("%zu\\n", sizeof(lbm_timing));')
    prog += [f'printf("%zu\\n", offsetof(lbm_timing, {f}));' for f in tfields]
    prog.append('printf("%zu\\n", sizeof(lbm_schedule));')
    prog += [f'printf("%zu\\n", offsetof(lbm_schedule, {f}));' for f in sfields]
    prog.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(B.LbmConfig)] + [getattr(B.LbmConfig, f).offset for f in fields]
    want += [ctypes.sizeof(B.LbmTiming)] + [getattr(B.LbmTiming, f).offset for f in tfields]
    want += [ctypes.sizeof(B.LbmSchedule)] + [getattr(B.LbmSchedule, f).offset for f in sfields]
    assert got == want


def test_status_strings(lib):
    for s in range(7):
        assert B.status_string(s)
    assert B.status_string(99) == "unknown status"


def _cfg(**kw):
    case = I.small_channel(16, 8)
    return B.config_from_case(case, **kw)


@pytest.mark.parametrize("field,value", [
    ("tau", 0.5), ("lattice", 7), ("nz", 0), ("window_len", 0), ("sample_every", 3),
    ("ckpt_every", 7), ("g_max", 1.5), ("precision", 5), ("rho_out", -1.0),
    ("objective_kind", 9), ("q_interp", 0.0), ("ckpt_format", 4),
])
def test_invalid_configs_are_rejected(lib, field, value):
    cfg = _cfg()
    setattr(cfg, field, value)
    with pytest.raises(B.LbmError) as e:
        B.workspace_size(cfg)
    assert e.value.status == B.LBM_ERR_ARG
    assert B.last_error()


def test_d2q9_batches_are_valid_configs(lib):
    """nz > 1 with D2Q9 stacks independent 2D lattices (a batch)."""
    cfg = _cfg()
    cfg.nz = 5
    assert B.workspace_size(cfg) > B.workspace_size(_cfg())


def test_sixteen_bit_checkpoints_need_fp32(lib):
    cfg = _cfg(precision=B.LBM_FP64)
    cfg.ckpt_format = 1
    with pytest.raises(B.LbmError):
        B.workspace_size(cfg)


@pytest.mark.parametrize("lattice", [9, 19])
def test_moment_checkpoints_are_smaller_and_allowed_in_fp64(lib, lattice):
    """Checkpoints 1..S-1 keep 7 (2D) / 11 (3D) coefficient planes instead of
    Q; checkpoint 0 stays native.  The format is lossless, so FP64 may use it."""
    case = I.small_channel(64, 12, window_len=40, ckpt_every=4) if lattice == 9 else \
        I.small_duct3d(32, 8, 8, window_len=40, ckpt_every=4)
    sizes = {}
    for fmt in (I.CKPT_NATIVE, I.CKPT_MOMENT):
        cfg = B.config_from_case(case.replace(ckpt_format=fmt))
        sizes[fmt] = B.workspace_size(cfg)
    n, S, R = case.n, 10, 4
    saved = (S - 1) * (lattice - (7 if lattice == 9 else 11)) * n * R   # checkpoint planes saved
    extra = n * R * lattice                                                # one more segment slot (K, not K-1)
    assert sizes[I.CKPT_NATIVE] - sizes[I.CKPT_MOMENT] == pytest.approx(saved - extra, abs=4096 * 12)
    cfg = B.config_from_case(case.replace(ckpt_format=I.CKPT_MOMENT), precision=B.LBM_FP64)
    assert B.workspace_size(cfg) > 0


def test_bad_box_rejected(lib):
    cfg = _cfg()
    cfg.design_box[1] = 99
    with pytest.raises(B.LbmError):
        B.workspace_size(cfg)


def test_workspace_grows_with_segment_length(lib):
    a = B.workspace_size(_cfg())
    cfg = _cfg()
    cfg.ckpt_every = 10
    b = B.workspace_size(cfg)
    cfg.ckpt_every = 1
    c = B.workspace_size(cfg)
    assert a > b and c > 0


def _create(case, cls=None, **kw):
    cfg = B.config_from_case(case, **kw)
    cls = case.node_class.reshape(-1).astype(np.uint8) if cls is None else cls
    gam = case.gamma.reshape(-1).astype(np.float32)
    ctx = ctypes.c_void_p()
    st = B.lib().lbm_create(ctypes.byref(cfg), cls.ctypes.data, gam.ctypes.data, None, None,
                            None, 0, None, ctypes.byref(ctx))
    return st


def test_create_rejects_bad_node_classes_on_the_host(lib):
    case = I.small_channel(16, 8)
    cls = case.node_class.reshape(-1).astype(np.uint8).copy()
    bad = cls.copy()
    bad[3 * 16 + 5] = I.WALL            # interior node must be FLUID
    assert _create(case, bad) == B.LBM_ERR_ARG
    bad = cls.copy()
    bad[3 * 16 + 15] = I.INLET          # inlet on the east face
    assert _create(case, bad) == B.LBM_ERR_ARG
    bad = cls.copy()
    bad[0] = I.INLET                    # inlet on a corner
    assert _create(case, bad) == B.LBM_ERR_ARG
    bad = cls.copy()
    bad[3 * 16 + 0] = I.FLUID           # boundary node with unknowns
    assert _create(case, bad) == B.LBM_ERR_ARG
    bad = cls.copy()
    bad[3 * 16 + 0] = 9                 # unknown class
    assert _create(case, bad) == B.LBM_ERR_ARG


def test_create_rejects_a_missing_workspace(lib):
    case = I.small_channel(16, 8)
    assert _create(case) == B.LBM_ERR_WORKSPACE


def test_pressure_outlet_is_d2q9_only(lib):
    case = I.small_duct3d(8, 5, 5, outlet=I.OUTLET_P)
    assert _create(case) == B.LBM_ERR_ARG


def test_mma_workspace_size_and_arguments_on_the_host(lib):
    """lbm_mma_workspace_size validates n and m before any CUDA call, and
    grows with n and m (the approximation coefficients are [m+1][n] each);
    lbm_mma_create rejects null pointers the same way."""
    size = ctypes.c_size_t()
    for n, m in ((0, 1), (10, 0), (10, B.LBM_MMA_MAX_M + 1)):
        assert lib.lbm_mma_workspace_size(n, m, ctypes.byref(size)) == B.LBM_ERR_ARG
    sizes = {}
    for n, m in ((1000, 1), (1000, 2), (2000, 2)):
        assert lib.lbm_mma_workspace_size(n, m, ctypes.byref(size)) == B.LBM_OK
        assert size.value % 256 == 0
        sizes[n, m] = size.value
    # per variable: 8 vectors of n doubles + p and q for every function (each region rounded to 256 bytes)
    assert abs((sizes[1000, 2] - sizes[1000, 1]) - 2 * 1000 * 8) <= 2 * 256
    assert abs((sizes[2000, 2] - sizes[1000, 2]) - (8 + 2 * 3) * 1000 * 8) <= 10 * 256
    h = ctypes.c_void_p()
    assert lib.lbm_mma_create(10, 1, None, None, None, 0, None, ctypes.byref(h)) == B.LBM_ERR_ARG
    assert lib.lbm_mma_update(None, None, None, None, None) == B.LBM_ERR_ARG


def test_every_workload_is_a_valid_configuration(lib):
    """Each shipped workload passes the host-side validation of lbm_workspace_size
    (FP32, and FP64 with native checkpoints); the full-time form of the cylinder
    case (a 60000-step window kept whole, K = 1) sizes to its complete history."""
    for name, make in I.WORKLOADS.items():
        case = make()
        n = B.workspace_size(B.config_from_case(case, B.LBM_FP32, pipeline=1))
        assert n > case.n * case.lattice * 4 * 2, name
        n64 = B.workspace_size(B.config_from_case(case.replace(ckpt_format=I.CKPT_NATIVE), B.LBM_FP64))
        assert n64 > 0, name
    cyl = I.WORKLOADS["cylinder200x100"]()
    T = 12 * cyl.window_len
    full = cyl.replace(window_len=T, ckpt_every=1, sample_from=T - cyl.window_len)
    size = B.workspace_size(B.config_from_case(full, B.LBM_FP32, pipeline=1))
    history = T * cyl.n * cyl.lattice * 4
    assert history <= size <= history * 1.01 + (1 << 28)
