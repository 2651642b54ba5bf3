"""Planted mistakes in the oracle must fail its pins.

Each case patches one plausible mistake into the oracle (a dropped term, a
wrong sign, a transposed operand, a wrong index) on the CPU and checks that the
corresponding pin in test_oracle_pins would reject it.  Nothing here touches a
GPU or the library.
"""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2608_19617_b300 import inputs as I


def _cs_gap(pr, p0):
    """Relative gap between the adjoint and the complex-step derivative."""
    traj = pr.run_window(p0)[3]
    _, dgamma, _ = pr.adjoint_window(traj)
    d = np.random.default_rng(5).standard_normal(pr.n)
    h = 1e-30
    want = pr.window_objective(p0.astype(complex), pr.case.gamma.reshape(-1) + 1j * h * d).imag / h
    return abs(dgamma @ d - want) / abs(want)


@pytest.fixture(scope="module")
def setup():
    case = I.small_channel(10, 7, obj_kind=I.OBJ_DISSIPATION, window_len=6, outlet=I.OUTLET_P,
                           profile="parabolic")
    pr = O.Problem(case)
    p0 = pr.initial_state()
    g = pr.g()
    for _ in range(25):
        _, _, p0, _ = pr.step(p0, g)
    return pr, p0


def test_unmutated_gap_is_rounding(setup):
    pr, p0 = setup
    assert _cs_gap(pr, p0) < 1e-10


def test_dropped_tau_term_is_caught(setup, monkeypatch):
    pr, p0 = setup
    orig = O.Problem.local_jacobian

    def mutant(self, f, h, aux, g):
        _, ja = orig(self, f, h, aux, g)
        dh = ja["dh"] - aux["hneq"][:, None, :] * ja["dtau"][None] / aux["tau_eff"] ** 2
        return dh + g[None, None] * (dh[self.lat.opp] - dh), ja

    monkeypatch.setattr(O.Problem, "local_jacobian", mutant)
    assert _cs_gap(pr, p0) > 1e-6


def test_transposed_jacobian_is_caught(setup, monkeypatch):
    pr, p0 = setup
    orig = O.Problem.local_jacobian

    def mutant(self, f, h, aux, g):
        jac, ja = orig(self, f, h, aux, g)
        return np.swapaxes(jac, 0, 1), ja

    monkeypatch.setattr(O.Problem, "local_jacobian", mutant)
    assert _cs_gap(pr, p0) > 1e-6


def test_wrong_sign_of_sensitivity_is_caught(setup, monkeypatch):
    pr, p0 = setup
    monkeypatch.setattr(O, "dg_dphi", lambda phi, q, gm: gm * q * (1 + q) / (phi + q) ** 2)
    assert _cs_gap(pr, p0) > 1e-6


def test_untransposed_boundary_adjoint_is_caught(setup, monkeypatch):
    pr, p0 = setup
    monkeypatch.setattr(O.Problem, "stream_adjoint",
                        lambda self, b: (self.S @ b.reshape(-1)).reshape(b.shape))
    assert _cs_gap(pr, p0) > 1e-6


def test_wrong_zouhe_index_is_caught(monkeypatch):
    """Swapping f2/f4 in the inlet rule for f5 breaks the inlet moment pin."""
    orig = O.Problem._boundary_rule

    def mutant(self, i, unk, fk, src):
        out = orig(self, i, unk, fk, src)
        if int(self.cls[i]) == O.INLET:
            u0 = float(self.case.inlet_u.reshape(-1)[i // self.nx])
            rho = (fk[0] + fk[2] + fk[4] + 2.0 * (fk[3] + fk[6] + fk[7])) * (1.0 / (1.0 - u0))
            out[5] = fk[7] + (fk[2] - fk[4]) * 0.5 + rho * (u0 / 6.0)
        return out

    monkeypatch.setattr(O.Problem, "_boundary_rule", mutant)
    case = I.small_channel(8, 6, u_in=0.06)
    pr = O.Problem(case)
    rng = np.random.default_rng(1)
    p = pr.initial_state() + 0.01 * pr.lat.w[:, None] * rng.standard_normal((9, pr.n))
    f = pr.stream(p)
    rho, u = O.moments_of(pr.lat, f)
    inl = case.node_class.reshape(-1) == I.INLET
    assert np.abs(u[1, inl]).max() > 1e-6


def test_dropped_cs2_delta_in_regularization_is_caught():
    """Without the -cs^2 delta term the regularized part gains mass."""
    lat = O.Lattice(9)
    rng = np.random.default_rng(2)
    f = O.equilibrium(lat, np.ones(20), 0.05 * rng.standard_normal((2, 20)))
    f = f + 0.02 * lat.w[:, None] * rng.standard_normal((9, 20))
    h, aux = O.collide(lat, f, 0.52, 0.1)
    wrong = lat.w[:, None] / (2 * O.CS4) * np.einsum("ap,aq,pqn->an", lat.c, lat.c, aux["pi"])
    assert np.abs(wrong.sum(0)).max() > 1e-4
    assert np.abs(aux["hneq"].sum(0)).max() < 1e-15


def _closed_form_gap(q=9, window_len=12, sample_every=3, sample_from=3):
    from _util import decaying_stream_window
    J, M, J_want, M_want = decaying_stream_window(q, window_len, sample_every, sample_from)
    return max(abs(J - J_want) / abs(J_want), abs(M - M_want) / abs(M_want))


def test_unmutated_closed_form_gap_is_rounding():
    assert _closed_form_gap() < 1e-13


def test_dropped_half_in_drag_coefficient_is_caught(monkeypatch):
    """Eq. 25 without the 1/2 of the dynamic pressure."""
    def mutant(self, f, h, aux, g):
        j = (self.w_obj * self.local_objective(f, h, aux, g)).sum()
        c = self.case
        return j, self.drag_density(h, g).sum() / (c.rho_out * c.monitor_u ** 2 * c.monitor_l)

    monkeypatch.setattr(O.Problem, "sample", mutant)
    assert _closed_form_gap() > 0.1


def test_weight_ignoring_the_first_sampled_step_is_caught(monkeypatch):
    """Eq. 42 weight dW/|W| instead of dW over the sampled span."""
    monkeypatch.setattr(O.Problem, "sample_weight",
                        lambda self: int(self.case.sample_every) / int(self.case.window_len))
    assert _closed_form_gap() > 0.1


def test_sampling_every_step_is_caught(monkeypatch):
    """Samples at every step of the span instead of every dW-th step."""
    monkeypatch.setattr(O.Problem, "sampled", lambda self, k: k >= int(self.case.sample_from))
    assert _closed_form_gap() > 1e-3


def test_shifted_sampling_instants_are_caught(monkeypatch):
    """Samples one step late (k = s0 + 1, s0 + 1 + dW, ...)."""
    def mutant(self, k):
        s0, dw = int(self.case.sample_from), int(self.case.sample_every)
        return k > s0 and (k - s0 - 1) % dw == 0

    monkeypatch.setattr(O.Problem, "sampled", mutant)
    assert _closed_form_gap() > 1e-3
