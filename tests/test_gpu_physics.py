"""Physics checks of the CUDA path at the paper's own sizes (too slow for the
CPU oracle), through the C ABI:

  * capillary wave, 256 x 512, lambda = 256, W = 4, M = 0.02, equal
    viscosities nu = 0.005 (Sec. 5.1): the interface amplitude follows the
    repaired Prosperetti solution over 1.5 periods;
  * 3D stationary drop, 100^3 periodic, R = 25, sigma = 1e-3, W = 4,
    rho* = 1000 (Sec. 5.2, tab:laplace_errors reports 0.31-1.04 %):
    Laplace's law dp = 2 sigma / R in 3D.
"""
import numpy as np
import pytest

import lbm_cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_12205_gb300 import build, lbm
    build.build()
    lbm.load()
    return lbm


def test_capillary_wave_vs_prosperetti(lib, report):
    pytest.importorskip("scipy")
    from prosperetti import amplitude
    L, sigma, nu = 256, 1e-3, 0.005
    p, phi, u, ps = C.capillary_wave2d(L=L, amp=0.01 * L, sigma=sigma, rho_ratio=1.0, nu=nu, W=4.0)
    sim = lib.LBM(p)
    sim.init_fields(phi, u, ps)
    k = 2 * np.pi / L
    om0 = np.sqrt(sigma * k ** 3 / 2.0)
    T = 2 * np.pi / om0
    nsamp, dt = 60, int(1.5 * T / 60)

    def eta():
        ph = sim.fields()[0][0][:, L // 2].astype(np.float64)
        s = ph - 0.5
        j = np.where((s[:-1] > 0) & (s[1:] <= 0))[0][0]
        return j + s[j] / (s[j] - s[j + 1]) - L
    e0 = eta()
    ts, es = [], []
    for i in range(nsamp):
        sim.step(dt)
        ts.append((i + 1) * dt)
        es.append(eta() / e0)
    ref = amplitude(np.array(ts, float), k, nu, sigma, 1.0, 1.0)
    dev = np.abs(np.array(es) - ref).max()
    report("capillary_wave_L256", max_dev=dev, omega0=om0, steps=nsamp * dt)
    assert dev < 0.05


def test_laplace_3d_drop(lib, report):
    R, sigma = 25.0, 1e-3
    p, phi, u, ps = C.drop3d(n=100, R=R, sigma=sigma, W=4.0, tau_H=0.5)
    sim = lib.LBM(p)
    sim.init_fields(phi, u, ps)
    sim.step(20000)
    d = sim.diag(1e-3)
    dp = d["sum_p_in"] / d["n_in"] - d["sum_p_out"] / d["n_out"]
    err = dp / (2 * sigma / R) - 1
    report("laplace_3d_R25", rel_err=err, dp=dp, mass=d["sum_phi"])
    assert d["finite"] == 1
    assert abs(err) < 0.03
