"""Host logic of the optimization loop (Alg. 2) without a GPU: the beta
schedule, the scaling of the objective and of the volume band handed to MMA,
and the termination on the relative change of J_eff.  The solver and the MMA
run are replaced by recording fakes; their device work is tested in
test_gpu_mma.py."""
import numpy as np
import pytest

from paper_2608_19617_b300 import inputs as I
from paper_2608_19617_b300 import optimize as OPT


class FakeTensor:
    def __init__(self, a):
        self.a = np.asarray(a, np.float64)

    def float(self):
        return self

    def contiguous(self):
        return self

    def cpu(self):
        return self

    def numpy(self):
        return self.a


class FakeSolver:
    """J_eff follows a scripted sequence; volume = mean of the raw design in the box."""

    def __init__(self, case, precision, js, vol):
        self.case, self.js, self.vol = case, list(js), vol
        self.device, self.stream = "cpu", None
        self.betas, self.closed = [], False

    def set_design_filtered(self, x, radius, beta, eta):
        self.betas.append(beta)
        self.x = x.a.copy()

    def run_until_converged(self, max_windows=None):
        return [dict(J=0.0, M=0.0, ratio=1.0, converged=False), dict(J=0.0, M=0.0, ratio=1e-4, converged=True)]

    def adjoint_window(self):
        return self.js.pop(0)

    def design_gradient_filtered(self):
        return np.full(self.case.n, 2.0)

    def design_volume(self):
        return self.vol

    def filter_chain_rule(self, dg):
        return dg * 3.0

    def close(self):
        self.closed = True


class FakeMma:
    calls = []

    def __init__(self, xmin, xmax, m, device=None, stream=None):
        assert m == 2 and np.all(xmin == 0) and np.all(xmax == 1)
        self.closed = False

    def update(self, x, fval, dfdx):
        FakeMma.calls.append((np.array(fval), np.array(dfdx)))
        return np.array([0.5, 0.0])

    def close(self):
        self.closed = True


@pytest.fixture
def fakes(monkeypatch):
    import torch
    made = {}

    def solver(case, precision):
        made["sol"] = FakeSolver(case, precision, made["js"], made["vol"])
        return made["sol"]

    monkeypatch.setattr(OPT.B, "Solver", solver)
    monkeypatch.setattr(OPT.B, "Mma", FakeMma)
    monkeypatch.setattr(torch, "tensor", lambda a, device=None: FakeTensor(a))
    FakeMma.calls = []
    return made


def test_beta_schedule_scaling_and_iteration_count(fakes):
    case = I.small_channel(20, 10, window_len=10)
    fakes["js"], fakes["vol"] = [2.0, 1.5, 1.2, 1.0, 0.9, 0.85, 0.8], 0.5
    hist, x = OPT.optimize(case, n_max=7, eps_o=0.0, vmin=0.4, vmax=0.45, beta_every=2, beta_max=6.0)
    assert [h["beta"] for h in hist] == [2, 2, 4, 4, 6, 6, 6]
    assert fakes["sol"].closed
    mask = OPT.design_mask(case)
    nd = mask.sum()
    f, df = FakeMma.calls[0]
    # objective scaled by |J| of the first iteration; band as V/Vmax - 1 and 1 - V/Vmin
    assert f[0] == pytest.approx(1.0) and f[1] == pytest.approx(0.5 / 0.45 - 1) and f[2] == pytest.approx(1 - 0.5 / 0.4)
    assert np.allclose(df[0], 2.0 / 2.0)
    assert np.allclose(df[1], 3.0 * mask / nd / 0.45) and np.allclose(df[2], -3.0 * mask / nd / 0.4)
    f, _ = FakeMma.calls[3]
    assert f[0] == pytest.approx(1.0 / 2.0)           # J = 1.0 over the first |J| = 2.0
    assert hist[-1]["converged"] and hist[0]["windows"] == 2


def test_stops_on_the_relative_change_of_j(fakes):
    case = I.small_channel(20, 10, window_len=10)
    fakes["js"], fakes["vol"] = [1.0, 0.9, 0.8999, 0.5, 0.4], 0.5
    hist, _ = OPT.optimize(case, n_max=5, eps_o=5e-3, vmin=0.4, vmax=0.45)
    assert len(hist) == 3                     # |0.8999 - 0.9| <= 5e-3 * 0.8999
