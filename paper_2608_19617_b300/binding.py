"""ctypes binding of liblbmadj.so: the C ABI of include/lbmadj.h, one Python
function per C function, plus a small ``Solver`` wrapper that owns a context
and its device workspace (a torch uint8 tensor).

This module only marshals arguments.  Every step of the solver runs in the
CUDA library; there is no fallback: if the library cannot be loaded the
import of a solver raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int32, c_int64, c_size_t, c_uint8, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbmadj.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_WORKSPACE, LBM_ERR_CUDA, LBM_ERR_STATE, LBM_ERR_NONFINITE, LBM_NOT_CONVERGED = range(7)
LBM_FP32, LBM_FP64 = 0, 1
LBM_MMA_MAX_M = 8
NUM_PHASES = 4
PHASES = ("forward", "recompute", "adjoint", "checkpoint")


class LbmConfig(ctypes.Structure):
    _fields_ = [
        ("lattice", c_int32), ("nx", c_int32), ("ny", c_int32), ("nz", c_int32),
        ("precision", c_int32), ("periodic", c_int32 * 3),
        ("tau", c_double), ("cs_smag", c_double), ("q_interp", c_double), ("g_max", c_double),
        ("rho_out", c_double),
        ("objective_kind", c_int32), ("monitor_kind", c_int32),
        ("objective_uref", c_double * 3), ("monitor_u", c_double), ("monitor_l", c_double),
        ("window_len", c_int32), ("sample_every", c_int32), ("conv_tol", c_double),
        ("ckpt_every", c_int32), ("ckpt_format", c_int32),
        ("obj_box", c_int32 * 6), ("design_box", c_int32 * 6), ("pipeline", c_int32),
    ]


class LbmTiming(ctypes.Structure):
    _fields_ = [("ms", c_double * NUM_PHASES), ("launches", c_int64 * NUM_PHASES),
                ("lattice_updates", c_int64 * NUM_PHASES)]


class LbmFilter(ctypes.Structure):
    _fields_ = [("radius", c_double), ("beta", c_double), ("eta", c_double)]


class LbmSchedule(ctypes.Structure):
    _fields_ = [("graphs", c_int32), ("pdl", c_int32),
                ("kernels_window", c_int64), ("kernels_adjoint", c_int64)]


class LbmError(RuntimeError):
    def __init__(self, status, func, msg):
        super().__init__(f"{func}: {status_string(status)} ({msg})")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Load liblbmadj.so (built by paper_2608_19617_b300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2608_19617_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    st = c_int32
    sig = {
        "lbm_workspace_size": (st, [POINTER(LbmConfig), POINTER(c_size_t)]),
        "lbm_create": (st, [POINTER(LbmConfig), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                            c_void_p, POINTER(c_void_p)]),
        "lbm_step_window": (st, [c_void_p, POINTER(c_double), POINTER(c_double)]),
        "lbm_window_converged": (st, [c_void_p, POINTER(c_int32), POINTER(c_double)]),
        "lbm_step_window_along": (st, [c_void_p, c_void_p, POINTER(c_double), POINTER(c_double)]),
        "lbm_window_objectives": (st, [c_void_p, c_void_p, c_void_p, c_size_t]),
        "lbm_adjoint_window": (st, [c_void_p, POINTER(c_double)]),
        "lbm_design_gradient": (st, [c_void_p, c_void_p, c_size_t]),
        "lbm_set_design": (st, [c_void_p, c_void_p]),
        "lbm_set_design_filtered": (st, [c_void_p, c_void_p, POINTER(LbmFilter)]),
        "lbm_design_gradient_filtered": (st, [c_void_p, c_void_p, c_size_t]),
        "lbm_get_design": (st, [c_void_p, c_void_p, c_size_t]),
        "lbm_get_state": (st, [c_void_p, c_void_p, c_size_t]),
        "lbm_set_state": (st, [c_void_p, c_void_p, c_size_t]),
        "lbm_get_adjoint_state": (st, [c_void_p, c_void_p, c_size_t]),
        "lbm_advance": (st, [c_void_p, c_int32]),
        "lbm_set_timing": (st, [c_void_p, c_int32]),
        "lbm_get_timing": (st, [c_void_p, POINTER(LbmTiming)]),
        "lbm_get_counters": (st, [c_void_p, POINTER(c_int64), POINTER(c_int64)]),
        "lbm_set_graphs": (st, [c_void_p, c_int32]),
        "lbm_set_pdl": (st, [c_void_p, c_int32]),
        "lbm_set_sample_start": (st, [c_void_p, c_int32]),
        "lbm_filter_chain_rule": (st, [c_void_p, c_void_p, c_void_p, c_size_t]),
        "lbm_design_volume": (st, [c_void_p, POINTER(c_double)]),
        "lbm_mma_workspace_size": (st, [c_size_t, c_int32, POINTER(c_size_t)]),
        "lbm_mma_create": (st, [c_size_t, c_int32, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p,
                                POINTER(c_void_p)]),
        "lbm_mma_update": (st, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
        "lbm_mma_destroy": (st, [c_void_p]),
        "lbm_get_schedule": (st, [c_void_p, POINTER(LbmSchedule)]),
        "lbm_run_until_converged": (st, [c_void_p, c_int32, POINTER(c_int32), POINTER(c_double), POINTER(c_double),
                                         POINTER(c_double)]),
        "lbm_step_window_noalloc": (st, [POINTER(LbmConfig), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p, POINTER(c_double), POINTER(c_double)]),
        "lbm_status_string": (ctypes.c_char_p, [c_int32]),
        "lbm_last_error": (ctypes.c_char_p, []),
        "lbm_destroy": (None, [c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def status_string(s: int) -> str:
    return lib().lbm_status_string(s).decode()


def last_error() -> str:
    return lib().lbm_last_error().decode()


def check(status: int, func: str):
    if status != LBM_OK:
        raise LbmError(status, func, last_error())


def config_from_case(case, precision=LBM_FP32, **overrides) -> LbmConfig:
    """Fill an lbm_config from an ``inputs.Case``."""
    c = LbmConfig()
    c.lattice, c.nx, c.ny, c.nz = case.lattice, case.nx, case.ny, case.nz
    c.precision = precision
    for k in range(3):
        c.periodic[k] = int(case.periodic[k])
        c.objective_uref[k] = float(case.obj_uref[k])
    c.tau, c.cs_smag, c.q_interp, c.g_max, c.rho_out = (float(case.tau), float(case.cs_smag),
                                                        float(case.q_interp), float(case.g_max),
                                                        float(case.rho_out))
    c.objective_kind, c.monitor_kind = int(case.obj_kind), int(case.monitor_kind)
    c.monitor_u, c.monitor_l = float(case.monitor_u), float(case.monitor_l)
    c.window_len, c.sample_every, c.conv_tol = int(case.window_len), int(case.sample_every), float(case.conv_tol)
    c.ckpt_every, c.ckpt_format = int(case.ckpt_every), int(case.ckpt_format)
    for k in range(6):
        c.obj_box[k] = int(case.obj_box[k])
        c.design_box[k] = int(case.design_box[k])
    c.pipeline = 0
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def workspace_size(cfg: LbmConfig) -> int:
    n = c_size_t()
    check(lib().lbm_workspace_size(byref(cfg), byref(n)), "lbm_workspace_size")
    return n.value


def _ptr(x):
    """Address of a numpy array or torch tensor (host or device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


class Solver:
    """One lbm_ctx plus the torch tensor that backs its device workspace."""

    def __init__(self, case, precision=LBM_FP32, device="cuda", stream=None, **overrides):
        import torch

        self.case = case
        self.cfg = config_from_case(case, precision, **overrides)
        self.n = case.nx * case.ny * case.nz
        self.q = case.lattice
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        size = workspace_size(self.cfg)
        self.workspace = torch.empty(size, dtype=torch.uint8, device=self.device)
        cls = np.ascontiguousarray(case.node_class.reshape(-1), dtype=np.uint8)
        gam = np.ascontiguousarray(case.gamma.reshape(-1), dtype=np.float32)
        w = np.ascontiguousarray(case.obj_weights.reshape(-1), dtype=np.float32)
        uin = np.ascontiguousarray(case.inlet_u.reshape(-1), dtype=np.float32)
        ctx = c_void_p()
        check(lib().lbm_create(byref(self.cfg), _ptr(cls), _ptr(gam), _ptr(w), _ptr(uin),
                               self.workspace.data_ptr(), size, c_void_p(self.stream.cuda_stream),
                               byref(ctx)), "lbm_create")
        self.ctx = ctx
        if int(getattr(case, "sample_from", 0)):
            self.set_sample_start(case.sample_from)

    # -- C calls --------------------------------------------------------------
    def step_window(self):
        j, m = c_double(), c_double()
        check(lib().lbm_step_window(self.ctx, byref(j), byref(m)), "lbm_step_window")
        return j.value, m.value

    def step_window_along(self, ref):
        """One window along the trajectory of another solver's last window
        (lbm_step_window_along): each segment starts from ref's checkpoint."""
        j, m = c_double(), c_double()
        check(lib().lbm_step_window_along(self.ctx, ref.ctx, byref(j), byref(m)), "lbm_step_window_along")
        return j.value, m.value

    def window_converged(self):
        c, r = c_int32(), c_double()
        check(lib().lbm_window_converged(self.ctx, byref(c), byref(r)), "lbm_window_converged")
        return bool(c.value), r.value

    def window_objectives(self):
        """Per-slice window means (J, monitor) of a D2Q9 batch."""
        J = np.empty(self.case.nz, np.float64)
        M = np.empty(self.case.nz, np.float64)
        check(lib().lbm_window_objectives(self.ctx, J.ctypes.data, M.ctypes.data, self.case.nz),
              "lbm_window_objectives")
        return J, M

    def adjoint_window(self):
        j = c_double()
        check(lib().lbm_adjoint_window(self.ctx, byref(j)), "lbm_adjoint_window")
        return j.value

    def design_gradient(self, out=None):
        """dJ/dgamma (FP64 [N]) into ``out`` (numpy or torch, host or device)."""
        if out is None:
            out = np.empty(self.n, np.float64)
        check(lib().lbm_design_gradient(self.ctx, _ptr(out), self.n), "lbm_design_gradient")
        return out

    def set_design(self, gamma):
        if isinstance(gamma, np.ndarray):
            gamma = np.ascontiguousarray(gamma.reshape(-1), dtype=np.float32)
        check(lib().lbm_set_design(self.ctx, _ptr(gamma)), "lbm_set_design")

    def set_design_filtered(self, x_raw, radius=4.0, beta=2.0, eta=0.5):
        """Design from raw variables through the density filter and Heaviside projection."""
        if isinstance(x_raw, np.ndarray):
            x_raw = np.ascontiguousarray(x_raw.reshape(-1), dtype=np.float32)
        f = LbmFilter(float(radius), float(beta), float(eta))
        check(lib().lbm_set_design_filtered(self.ctx, _ptr(x_raw), byref(f)), "lbm_set_design_filtered")

    def design_gradient_filtered(self, out=None):
        """dJ/dx for the raw variables of the last filtered design (FP64 [N])."""
        if out is None:
            out = np.empty(self.n, np.float64)
        check(lib().lbm_design_gradient_filtered(self.ctx, _ptr(out), self.n), "lbm_design_gradient_filtered")
        return out

    def get_design(self, out=None):
        if out is None:
            out = np.empty(self.n, np.float32)
        check(lib().lbm_get_design(self.ctx, _ptr(out), self.n), "lbm_get_design")
        return out

    def get_state(self, out=None):
        if out is None:
            out = np.empty((self.q, self.n), np.float64)
        check(lib().lbm_get_state(self.ctx, _ptr(out), self.q * self.n), "lbm_get_state")
        return out

    def set_state(self, f):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
        check(lib().lbm_set_state(self.ctx, _ptr(f), self.q * self.n), "lbm_set_state")

    def get_adjoint_state(self, out=None):
        if out is None:
            out = np.empty((self.q, self.n), np.float64)
        check(lib().lbm_get_adjoint_state(self.ctx, _ptr(out), self.q * self.n), "lbm_get_adjoint_state")
        return out

    def advance(self, nsteps: int):
        check(lib().lbm_advance(self.ctx, int(nsteps)), "lbm_advance")

    def set_timing(self, enable: bool):
        check(lib().lbm_set_timing(self.ctx, int(bool(enable))), "lbm_set_timing")

    def get_timing(self) -> dict:
        t = LbmTiming()
        check(lib().lbm_get_timing(self.ctx, byref(t)), "lbm_get_timing")
        return {PHASES[k]: dict(ms=t.ms[k], launches=t.launches[k], lattice_updates=t.lattice_updates[k])
                for k in range(NUM_PHASES)}

    def set_graphs(self, enable: bool):
        check(lib().lbm_set_graphs(self.ctx, int(bool(enable))), "lbm_set_graphs")

    def set_pdl(self, enable: bool):
        check(lib().lbm_set_pdl(self.ctx, int(bool(enable))), "lbm_set_pdl")

    def filter_chain_rule(self, dgamma, out=None):
        """(d gamma / d x)^T dgamma through the filter and projection (lbm_filter_chain_rule)."""
        dg = np.ascontiguousarray(dgamma, dtype=np.float64).reshape(-1)
        out = np.empty(self.n) if out is None else out
        check(lib().lbm_filter_chain_rule(self.ctx, _ptr(dg), _ptr(out), self.n), "lbm_filter_chain_rule")
        return out

    def design_volume(self) -> float:
        """Mean gamma over the design box, V of Sec. 3.3 (lbm_design_volume)."""
        v = c_double()
        check(lib().lbm_design_volume(self.ctx, byref(v)), "lbm_design_volume")
        return v.value

    def set_sample_start(self, first: int):
        """First sampled step of each following window (lbm_set_sample_start);
        a full-time run of T steps samples from T - |W|."""
        check(lib().lbm_set_sample_start(self.ctx, int(first)), "lbm_set_sample_start")

    def schedule(self) -> dict:
        """Launch configuration and kernels per window / adjoint sweep (lbm_get_schedule)."""
        out = LbmSchedule()
        check(lib().lbm_get_schedule(self.ctx, byref(out)), "lbm_get_schedule")
        return {f: getattr(out, f) for f, _ in LbmSchedule._fields_}

    def counters(self):
        s, w = c_int64(), c_int64()
        check(lib().lbm_get_counters(self.ctx, byref(s), byref(w)), "lbm_get_counters")
        return s.value, w.value

    def run_until_converged(self, max_windows=None):
        """Alg. 1 outer loop: windows until the test of Eq. 26 holds."""
        mw = int(max_windows or self.case.max_windows)
        rec = []
        for _ in range(mw):
            j, m = self.step_window()
            conv, ratio = self.window_converged()
            rec.append(dict(J=j, M=m, ratio=ratio, converged=conv))
            if conv:
                break
        return rec

    def run_windows(self, max_windows=None):
        """Alg. 1 outer loop in the library (lbm_run_until_converged): returns
        (windows run, J, monitor, ratio, converged)."""
        mw = int(max_windows or self.case.max_windows)
        w, J, M, r = c_int32(), c_double(), c_double(), c_double()
        st = lib().lbm_run_until_converged(self.ctx, mw, byref(w), byref(J), byref(M), byref(r))
        if st not in (LBM_OK, LBM_NOT_CONVERGED):
            check(st, "lbm_run_until_converged")
        return w.value, J.value, M.value, r.value, st == LBM_OK

    def close(self):
        if getattr(self, "ctx", None):
            lib().lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mma:
    """One MMA run (lbm_mma_*): n design variables on the device, m
    constraints f_i <= 0.  update() takes the point as a float64 CUDA tensor
    (changed in place), the values [m+1] and the gradients [m+1][n]."""

    def __init__(self, xmin, xmax, m: int, device="cuda", stream=None):
        import torch

        xmin = np.ascontiguousarray(xmin, dtype=np.float64).reshape(-1)
        xmax = np.ascontiguousarray(xmax, dtype=np.float64).reshape(-1)
        self.n, self.m = xmin.size, int(m)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        size = c_size_t()
        check(lib().lbm_mma_workspace_size(self.n, self.m, byref(size)), "lbm_mma_workspace_size")
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        h = c_void_p()
        check(lib().lbm_mma_create(self.n, self.m, _ptr(xmin), _ptr(xmax), self.workspace.data_ptr(), size.value,
                                   c_void_p(self.stream.cuda_stream), byref(h)), "lbm_mma_create")
        self.h = h

    def update(self, x, fval, dfdx):
        """One iteration; returns the subproblem's multipliers."""
        import torch

        assert x.is_cuda and x.dtype == torch.float64 and x.is_contiguous() and x.numel() == self.n
        fv = np.ascontiguousarray(fval, dtype=np.float64).reshape(-1)
        assert fv.size == self.m + 1
        df = torch.as_tensor(dfdx, dtype=torch.float64, device=self.device).contiguous()
        assert df.numel() == (self.m + 1) * self.n
        lam = (c_double * self.m)()
        check(lib().lbm_mma_update(self.h, x.data_ptr(), _ptr(fv), df.data_ptr(), lam), "lbm_mma_update")
        return np.array(lam[:])

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_mma_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
