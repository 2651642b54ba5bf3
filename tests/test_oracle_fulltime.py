"""Pins of the oracle's full-time adjoint run (Sec. 4.2.3).

The full-time comparison keeps the whole flow history from the initial time
and traces the adjoint back to it, while the objective is still the mean over
the final window.  In the oracle that run is one window of T steps whose
sampling starts at step s0 = T - |W| (``case.sample_from``).  These tests pin
it to what must hold:

* its objective and final state equal those of a plain window of T - s0 steps
  after s0 unsampled spin-up steps (the same samples, added in the same order);
* its gradient (design field and start field) equals the complex-step
  derivative of its own forward run, and central differences of single-node
  perturbations;
* planting a sampling offset that the forward and the adjoint disagree on
  breaks the complex-step pin; weighting the samples by the whole run breaks
  the spin-up identity.
"""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2608_19617_b300 import inputs as I


def _developed(pr, steps=25):
    from _util import initial_flow
    p = initial_flow(pr)
    g = pr.g()
    for _ in range(steps):
        _, _, p, _ = pr.step(p, g)
    return p


CASES = [
    ("diss-zouhe-every2", lambda: I.small_channel(10, 7, obj_kind=I.OBJ_DISSIPATION, window_len=12, sample_every=2,
                                                   outlet=I.OUTLET_P, profile="parabolic"), 4),
    ("veldev-zg-odd-start", lambda: I.small_channel(10, 7, obj_kind=I.OBJ_VELOCITY_DEV, window_len=11,
                                                     outlet=I.OUTLET_ZG), 5),
    ("drag-periodic", lambda: I.small_channel(9, 6, obj_kind=I.OBJ_DRAG, window_len=9, sample_every=3,
                                              periodic_x=True, g_max=0.9), 3),
    ("d3q19-duct", lambda: I.small_duct3d(6, 5, 5, window_len=6), 2),
]


@pytest.mark.parametrize("name,mk,s0", CASES, ids=[c[0] for c in CASES])
def test_full_time_objective_is_the_final_window_after_spinup(name, mk, s0):
    base = mk()
    T = base.window_len
    full = O.Problem(base.replace(sample_from=s0))
    p0 = _developed(full)
    p_end, J, M, _ = full.run_window(p0, store=False)

    win = O.Problem(base.replace(window_len=T - s0, sample_from=0))
    p = p0
    g = win.g()
    for _ in range(s0):
        _, _, p, _ = win.step(p, g)
    q_end, Jw, Mw, _ = win.run_window(p, store=False)
    assert J == Jw and M == Mw            # the same samples, in the same order
    assert np.array_equal(p_end, q_end)
    assert J != O.Problem(base).run_window(p0, store=False)[1]   # the offset matters


@pytest.mark.parametrize("name,mk,s0", CASES, ids=[c[0] for c in CASES])
def test_full_time_adjoint_matches_complex_step(name, mk, s0):
    """Design and start-field gradients of the full-time run against the
    complex-step derivative of its forward map (exact to rounding)."""
    case = mk().replace(sample_from=s0)
    pr = O.Problem(case)
    p0 = _developed(pr)
    traj = pr.run_window(p0)[3]
    _, dgamma, a0 = pr.adjoint_window(traj)
    rng = np.random.default_rng(11)
    h = 1e-30
    d = rng.standard_normal(pr.n)
    want = pr.window_objective(p0.astype(complex), case.gamma.reshape(-1) + 1j * h * d).imag / h
    assert abs(want) > 1e-12
    assert abs(dgamma @ d - want) <= 1e-10 * abs(want), (dgamma @ d, want)
    dp = rng.standard_normal(p0.shape) * pr.lat.w[:, None]
    want = pr.window_objective(p0 + 1j * h * dp, case.gamma.reshape(-1)).imag / h
    assert abs((a0 * dp).sum() - want) <= 1e-10 * abs(want)


def test_full_time_adjoint_matches_central_differences():
    """Single-node perturbations of gamma (the protocol of Sec. 4.2.1) on a
    full-time run: 14 steps, samples over the last 6."""
    case = I.small_channel(12, 8, obj_kind=I.OBJ_DISSIPATION, window_len=14).replace(sample_from=8)
    pr = O.Problem(case)
    p0 = _developed(pr, 30)
    _, dgamma, _ = pr.adjoint_window(pr.run_window(p0)[3])
    gam = case.gamma.reshape(-1)
    for node in (3 * 12 + 4, 4 * 12 + 7, 2 * 12 + 9):
        e = np.zeros(pr.n)
        e[node] = 1e-6
        fd = (pr.window_objective(p0, gam + e) - pr.window_objective(p0, gam - e)) / 2e-6
        assert abs(fd - dgamma[node]) <= 1e-6 * abs(dgamma[node]), (node, fd, dgamma[node])


def _gap(pr, p0):
    _, dgamma, _ = pr.adjoint_window(pr.run_window(p0)[3])
    d = np.random.default_rng(5).standard_normal(pr.n)
    h = 1e-30
    want = pr.window_objective(p0.astype(complex), pr.case.gamma.reshape(-1) + 1j * h * d).imag / h
    return abs(dgamma @ d - want) / abs(want)


@pytest.fixture(scope="module")
def fulltime():
    case = I.small_channel(10, 7, obj_kind=I.OBJ_DISSIPATION, window_len=10, sample_every=2,
                           outlet=I.OUTLET_P, profile="parabolic").replace(sample_from=4)
    pr = O.Problem(case)
    return pr, _developed(pr)


def test_unmutated_full_time_gap_is_rounding(fulltime):
    assert _gap(*fulltime) < 1e-10


def test_adjoint_sampling_from_the_first_step_is_caught(fulltime, monkeypatch):
    """An adjoint that injects its objective sources at the plain window's
    instants (k % dW == 0) while the forward samples from s0 on."""
    pr, p0 = fulltime
    orig_adj = O.Problem.adjoint_window

    def mutant(self, traj, gamma=None):
        saved = O.Problem.sampled
        O.Problem.sampled = lambda s, k: k % int(s.case.sample_every) == 0
        try:
            return orig_adj(self, traj, gamma)
        finally:
            O.Problem.sampled = saved

    monkeypatch.setattr(O.Problem, "adjoint_window", mutant)
    assert _gap(pr, p0) > 1e-6


def test_weight_of_the_whole_run_is_caught(fulltime, monkeypatch):
    """Weighting the samples by dW / T (the whole run) instead of dW / (T - s0)
    scales J and its gradient by the same factor, so the complex-step pin
    cannot see it; the spin-up identity does."""
    pr, p0 = fulltime
    monkeypatch.setattr(O.Problem, "sample_weight", lambda s: int(s.case.sample_every) / int(s.case.window_len))
    J = pr.run_window(p0, store=False)[1]
    win = O.Problem(pr.case.replace(window_len=6, sample_from=0))
    p = p0
    for _ in range(4):
        _, _, p, _ = win.step(p, win.g())
    assert J != win.run_window(p, store=False)[1]
