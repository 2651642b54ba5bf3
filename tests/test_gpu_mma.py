"""The MMA design update, the design volume and the filter chain rule on the
GPU (lbm_mma_*, lbm_design_volume, lbm_filter_chain_rule), against the
oracle, and a short run of the optimization loop of Alg. 2.

Tolerances: the library and the oracle solve the same strictly concave dual
by different methods.  The library runs projected Newton on the device sums
and reaches a projected dual gradient near 1e-14.  The oracle's bounded
quasi-Newton routine stops near 1e-9, where the dual's values no longer
resolve an ascent.  So the multipliers agree to 1e-6 relative and the new
points to 1e-7 absolute on variables in [0, 1]; an error in the method
itself moves them by orders of magnitude more.  Every iteration feeds both
the same point (the library's), so both keep the same history of iterates.
"""
import numpy as np
import pytest

from oracle import lbm as O
from oracle import mma as OM
from paper_2608_19617_b300 import binding as B
from paper_2608_19617_b300 import inputs as I
from paper_2608_19617_b300 import optimize as OPT

from _util import f32_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2608_19617_b300 import build
    build.build()
    B.lib()


def _problem(n, m, seed):
    """A smooth nonconvex objective and m linear constraints, both as means
    over the variables (values of order one, multipliers below the cost of
    the artificial variables)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.5, 2.0, n)
    d = rng.standard_normal(n)
    A = rng.uniform(0.0, 1.0, (m, n)) / n
    b = A.sum(axis=1) * rng.uniform(0.3, 0.5, m)

    def evaluate(x):
        f = np.concatenate([[np.sum(c / (x + 0.1) + d * np.sin(3 * x)) / n], A @ x - b])
        df = np.vstack([(-c / (x + 0.1) ** 2 + 3 * d * np.cos(3 * x)) / n, A])
        return f, df

    return evaluate


@pytest.mark.parametrize("n,m", [(1000, 1), (4097, 2), (200003, 3)])
def test_mma_iterations_match_the_oracle(n, m):
    import torch
    evaluate = _problem(n, m, seed=n + m)
    rng = np.random.default_rng(1)
    xmin, xmax = np.zeros(n), np.ones(n)
    x0 = rng.uniform(0.3, 0.7, n)
    gpu = B.Mma(xmin, xmax, m)
    ora = OM.MMA(xmin, xmax)
    x = torch.tensor(x0, dtype=torch.float64, device="cuda")
    for it in range(6):
        xh = x.cpu().numpy()
        f, df = evaluate(xh)
        want, lam_w = ora.update(xh, f, df)
        lam = gpu.update(x, f, df)
        got = x.cpu().numpy()
        assert np.abs(got - want).max() < 1e-7, (it, np.abs(got - want).max())
        assert np.allclose(lam, lam_w, rtol=1e-6, atol=1e-9), (it, lam, lam_w)
        assert np.all(lam < OM.C_ART)          # the artificial variables stay at zero
    gpu.close()


def test_mma_reaches_the_closed_form_optimum_on_the_gpu():
    import torch
    rng = np.random.default_rng(4)
    n, V = 5000, 0.3
    c = rng.uniform(1.0, 4.0, n)
    want = V * n * np.sqrt(c) / np.sqrt(c).sum()
    gpu = B.Mma(np.full(n, 1e-3), np.ones(n), 1)
    x = torch.full((n,), 0.5, dtype=torch.float64, device="cuda")
    for _ in range(40):
        xh = x.cpu().numpy()
        # objective as a mean, so that the multiplier (about 10) stays below the artificial variables' cost
        gpu.update(x, np.array([(c / xh).mean(), xh.mean() - V]), np.vstack([-c / xh ** 2 / n, np.full(n, 1.0 / n)]))
    got = x.cpu().numpy()
    assert np.abs(got - want).max() < 1e-6
    assert abs(got.mean() - V) < 1e-8
    gpu.close()


def test_mma_arguments():
    with pytest.raises(B.LbmError) as e:
        B.Mma(np.zeros(4), np.ones(4), 0)
    assert e.value.status == B.LBM_ERR_ARG
    with pytest.raises(B.LbmError) as e:
        B.Mma(np.zeros(4), np.ones(4), B.LBM_MMA_MAX_M + 1)
    assert e.value.status == B.LBM_ERR_ARG
    with pytest.raises(B.LbmError) as e:
        B.Mma(np.ones(4), np.ones(4), 1)          # xmin must be below xmax
    assert e.value.status == B.LBM_ERR_ARG


def test_mma_update_rejects_host_pointers():
    """x and dfdx are read by the kernels: host memory is an argument error,
    caught on the host before any launch."""
    import torch
    n = 64
    gpu = B.Mma(np.zeros(n), np.ones(n), 1)
    f = np.zeros(2)
    x_host, df_host = np.full(n, 0.5), np.zeros((2, n))
    assert B.lib().lbm_mma_update(gpu.h, x_host.ctypes.data, f.ctypes.data, df_host.ctypes.data, None) == B.LBM_ERR_ARG
    x = torch.full((n,), 0.5, dtype=torch.float64, device="cuda")
    assert B.lib().lbm_mma_update(gpu.h, x.data_ptr(), f.ctypes.data, df_host.ctypes.data, None) == B.LBM_ERR_ARG
    df = torch.zeros((2, n), dtype=torch.float64, device="cuda")
    df[0] = 1.0
    df[1] = 1.0 / n
    gpu.update(x, np.array([0.0, -0.1]), df)          # a valid call still works afterwards
    assert torch.all(x < 0.5)
    gpu.close()


def test_design_volume_and_filter_chain_rule_match_the_oracle():
    case = f32_inputs(I.small_channel(150, 12, window_len=12, outlet=I.OUTLET_P, tau=0.53))
    shape = (case.nz, case.ny, case.nx)
    x_raw = np.clip(I.minmax_noise(shape, 2.0, 5) * 0.9, 0, 1).astype(np.float32)
    radius, beta, eta = 3.0, 8.0, 0.5
    sol = B.Solver(case, B.LBM_FP64)
    sol.set_design_filtered(x_raw, radius, beta, eta)
    gam = sol.get_design().astype(np.float64).reshape(shape)
    x0, x1, y0, y1, z0, z1 = case.design_box
    assert abs(sol.design_volume() - gam[z0:z1, y0:y1, x0:x1].mean()) < 1e-13
    rng = np.random.default_rng(2)
    dg = rng.standard_normal(case.n)
    got = sol.filter_chain_rule(dg)
    want = O.filter_project_adjoint(x_raw.astype(np.float64), dg, shape, case.design_box, radius, beta, eta)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # the volume gradient through the chain rule, against central differences of the oracle's projection
    mask = OPT.design_mask(case)
    dv = sol.filter_chain_rule(mask / mask.sum())
    xr = x_raw.astype(np.float64).reshape(-1)
    for j in (3 * 150 + 40, 6 * 150 + 77, 9 * 150 + 120):
        e = np.zeros_like(xr)
        e[j] = 1e-6

        def vol(v):
            return O.filter_project(v, shape, case.design_box, radius, beta, eta).reshape(shape)[
                z0:z1, y0:y1, x0:x1].mean()

        fd = (vol(xr + e) - vol(xr - e)) / 2e-6
        assert abs(fd - dv[j]) <= 1e-6 * abs(dv[j]) + 1e-12
    sol.close()


def _loop_case():
    case = f32_inputs(I.small_channel(96, 32, obj_kind=I.OBJ_DRAG, window_len=200, sample_every=10,
                                      outlet=I.OUTLET_P, tau=0.6, noise_amp=0.2))
    case = case.replace(design_box=(24, 72, 6, 26, 0, 1), max_windows=8)
    gam0 = case.gamma.copy()
    gam0[0, 6:26, 24:72] = 0.3
    return case.replace(gamma=gam0)


def test_optimization_loop_brings_the_volume_into_the_band():
    """Alg. 2 on a small drag case at fixed beta = 2: the volume starts above
    the band (the projection of 0.3 is about 0.25) and the MMA steps bring it
    into 0.1 <= V <= 0.12."""
    hist, x = OPT.optimize(_loop_case(), n_max=6, eps_o=0.0, vmin=0.1, vmax=0.12, radius=2.0, beta_every=100)
    assert len(hist) == 6
    assert all(np.isfinite(h["J"]) for h in hist)
    assert hist[0]["volume"] > 0.2
    assert 0.1 - 2e-3 <= hist[-1]["volume"] <= 0.12 + 2e-3
    assert np.all((x >= 0) & (x <= 1))


def test_optimization_loop_doubles_beta_up_to_its_cap():
    hist, _ = OPT.optimize(_loop_case(), n_max=5, eps_o=0.0, vmin=0.1, vmax=0.12, radius=2.0, beta_every=2,
                           beta_max=8.0)
    assert [h["beta"] for h in hist] == [2, 2, 4, 4, 8]
