"""Pins of the oracle's density filter and Heaviside projection (Sec. 3.3)."""
import numpy as np
import pytest

from oracle import lbm as O


def test_filter_preserves_constants_and_is_local():
    shape, box = (1, 12, 15), (2, 13, 1, 11, 0, 1)
    F = O.filter_weights(shape, box, 4.0)
    np.testing.assert_allclose(F @ np.full(F.shape[0], 0.37), 0.37, rtol=1e-15)
    # weights are max(0, r - d): a node 4 cells away contributes nothing
    e = np.zeros(F.shape[0])
    e[5 + 15 * 5] = 1.0
    out = (F @ e).reshape(12, 15)
    assert out[5, 9] == 0.0 and out[5, 8] > 0.0 and out[9, 5] == 0.0
    # outside the box the field is untouched
    x = np.random.default_rng(0).random(F.shape[0])
    y = (F @ x).reshape(12, 15)
    np.testing.assert_array_equal(y[:, 0], x.reshape(12, 15)[:, 0])


def test_filter_weight_hand_value():
    """Interior node, radius 2 in 2D: the neighbours at distance 1 weigh 1,
    at sqrt 2 weigh 2 - sqrt 2, the centre 2; normalised."""
    shape, box = (1, 7, 7), (0, 7, 0, 7, 0, 1)
    F = O.filter_weights(shape, box, 2.0).toarray()
    i = 3 + 7 * 3
    tot = 2 + 4 * 1 + 4 * (2 - np.sqrt(2))
    assert F[i, i] == pytest.approx(2 / tot, rel=1e-15)
    assert F[i, i + 1] == pytest.approx(1 / tot, rel=1e-15)
    assert F[i, i + 8] == pytest.approx((2 - np.sqrt(2)) / tot, rel=1e-15)
    assert F[i, i + 2] == 0.0


def test_heaviside_limits():
    """H(0) = 0, H(1) = 1, H(eta) = tanh(b eta)/(tanh(b eta)+tanh(b(1-eta)))."""
    for beta in (2.0, 8.0, 16.0):
        assert O.heaviside(0.0, beta, 0.5) == pytest.approx(0.0, abs=1e-15)
        assert O.heaviside(1.0, beta, 0.5) == pytest.approx(1.0, rel=1e-15)
        assert O.heaviside(0.5, beta, 0.5) == pytest.approx(0.5, rel=1e-15)
    # steep beta approaches a step
    assert O.heaviside(0.4, 64.0, 0.5) < 1e-2 and O.heaviside(0.6, 64.0, 0.5) > 0.99
    x = np.linspace(0, 1, 11)
    h = 1e-30
    np.testing.assert_allclose(O.heaviside_derivative(x, 4.0, 0.3),
                               O.heaviside(x + 1j * h, 4.0, 0.3).imag / h, rtol=1e-14)


def test_filter_projection_chain_rule_matches_complex_step():
    shape, box = (1, 10, 13), (1, 12, 1, 9, 0, 1)
    rng = np.random.default_rng(3)
    x = rng.random(130)
    g = rng.standard_normal(130)
    dx = O.filter_project_adjoint(x, g, shape, box, 3.0, 4.0, 0.5)
    d = rng.standard_normal(130)
    h = 1e-30
    phys = O.filter_project(x + 1j * h * d, shape, box, 3.0, 4.0, 0.5)
    assert dx @ d == pytest.approx(g @ phys.imag / h, rel=1e-13)


def test_filter_3d():
    shape, box = (6, 7, 8), (1, 7, 1, 6, 1, 5)
    F = O.filter_weights(shape, box, 2.5)
    np.testing.assert_allclose(F @ np.ones(F.shape[0]), 1.0, rtol=1e-15)
    assert F.nnz > F.shape[0]
