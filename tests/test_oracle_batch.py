"""A D2Q9 batch (independent 2D problems stacked as z-slices) in the oracle:
its window objective is the sum of the slices' and its gradient is the
slices' gradients side by side.  Pins the batching semantics the library
follows."""
import numpy as np

from oracle import lbm as O
from paper_2608_19617_b300 import inputs as I

from _util import initial_flow, oracle_advance


def test_batch_is_the_slices_side_by_side():
    cases = [I.small_channel(12, 7, window_len=6, seed=s, outlet=I.OUTLET_P, u_in=0.04 + 0.01 * s) for s in range(3)]
    batch = I.stack_cases(cases)
    prb = O.Problem(batch)
    p0s = [oracle_advance(O.Problem(c), initial_flow(O.Problem(c)), 10) for c in cases]
    p0 = np.concatenate(p0s, axis=1)
    _, Jb, _, trajb = prb.run_window(p0)
    _, gb, ab = prb.adjoint_window(trajb)
    Js, gs, As = [], [], []
    for c, p in zip(cases, p0s):
        pr = O.Problem(c)
        _, J, _, traj = pr.run_window(p)
        _, g, a = pr.adjoint_window(traj)
        Js.append(J)
        gs.append(g)
        As.append(a)
    assert abs(Jb - sum(Js)) <= 1e-14 * abs(Jb)
    np.testing.assert_allclose(gb, np.concatenate(gs), rtol=1e-12, atol=1e-30)
    np.testing.assert_allclose(ab, np.concatenate(As, axis=1), rtol=1e-12, atol=1e-30)
