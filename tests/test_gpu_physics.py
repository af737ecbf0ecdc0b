"""Physics checks of the CUDA path at the paper's own sizes (too slow for the
CPU oracle), through the C ABI:

  * capillary wave, 256 x 512, lambda = 256, W = 4, M = 0.02, equal
    viscosities nu = 0.005 (Sec. 5.1): the period of the interface amplitude
    against the repaired Prosperetti solution;
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
    """Period of the standing wave over two periods against the repaired
    Prosperetti solution.  Measured: 4.1 % longer at W = 4 (2.1 % at W = 8,
    independent of lambda between 256 and 512): the phase-field interface of
    width W carries a slightly smaller dynamic surface tension.  Held to 6 %."""
    pytest.importorskip("scipy")
    from prosperetti import amplitude
    L, sigma, nu = 256, 1e-3, 0.005
    p, phi, u, ps = C.capillary_wave2d(L=L, amp=0.01 * L, sigma=sigma, rho_ratio=1.0, nu=nu, W=4.0)
    sim = lib.LBM(p)
    sim.init_fields(phi, u, ps)
    k = 2 * np.pi / L
    om0 = np.sqrt(sigma * k ** 3 / 2.0)
    T = 2 * np.pi / om0
    nsamp = 80
    dt = int(2.0 * T / nsamp)

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
    ts, es = np.array(ts, float), np.array(es)
    ref = amplitude(ts, k, nu, sigma, 1.0, 1.0)

    def period(y):
        cr = [ts[i] - y[i] * (ts[i + 1] - ts[i]) / (y[i + 1] - y[i])
              for i in range(len(y) - 1) if y[i] * y[i + 1] < 0]
        return 2 * np.mean(np.diff(cr))
    ratio = period(es) / period(ref)
    report("capillary_wave_L256", period_ratio=ratio, max_dev=np.abs(es - ref).max(), omega0=om0)
    assert abs(ratio - 1) < 0.06


def test_laplace_3d_drop(lib, report):
    """tab:laplace_errors at sigma = 1e-3: 100^3 periodic box, drops of
    R = 15 .. 35, W = 4, rho* = 1000, tau = 0.5, 50,000 iterations.
    eq:laplace_law takes R as the radius of the drop in its equilibrium
    state: here the radius of the sphere enclosing as many nodes as the
    phi > 1/2 region (the interface is phi = 1/2); dp = 2 sigma / R in 3D
    (reading R10).  The paper prints 0.91 % (R = 15) falling to 0.31 %
    (R = 35); this model's pressure jump is a few per cent low and, like the
    paper's, its error falls as the drop grows (about 1 / R)."""
    sigma = 1e-3
    errs = []
    for R in (15.0, 20.0, 25.0, 30.0, 35.0):
        p, phi, u, ps = C.drop3d(n=100, R=R, sigma=sigma, W=4.0, tau_H=0.5)
        sim = lib.LBM(p)
        sim.init_fields(phi, u, ps)
        sim.step(50000)
        d = sim.diag(1e-3)
        js = sim.jet_stats(0.5, 8)
        assert js["n_components"] == 1 and js["has_jet"] == 0      # one drop, clear of z = 0
        r_half = (3.0 * js["drop_volume"] / (4.0 * np.pi)) ** (1.0 / 3.0)
        err = d["dp_laplace"] / (2 * sigma / r_half) - 1
        report("laplace_3d_R%d" % int(R), rel_err=err, r_half=r_half, rel_err_initial_radius=d["dp_laplace"] / (2 * sigma / R) - 1,
               dp=d["dp_laplace"], mass=d["sum_phi"])
        assert d["finite"] == 1
        errs.append(err)
        sim.close()
    errs = np.abs(np.array(errs))
    assert errs.max() < 0.05
    # the error shrinks as the drop grows, like the paper's
    assert np.all(np.diff(errs) < 0.002) and errs[-1] < 0.7 * errs[0]


def test_poiseuille_converges_to_the_fd_solution(lib, report):
    """Layered two-phase Poiseuille flow (Sec. 5.3, rho* = 1000, mu* = 100,
    tau_H = 0.5), refined at a fixed ratio W / ny = 1/16 and g ~ 1/ny^2: the
    relative L2 error (eq:l2_norm_error) against a second-order FD solution of
    eq:momentum_equation with the solver's own rho(phi), mu(phi) falls at
    second order (the paper's slope -1.94) and reaches ~1e-3 at ny = 256.  The
    oracle checks the same at ny = 64 and 128 (too slow beyond).  (At ny = 512
    float32 stops the approach to the steady state: near it the per-step
    change of u falls below its rounding, a floor that grows like ny^2 --
    measured 2.1e-3 there.)"""
    from test_oracle_physics import fd_poiseuille
    errs = {}
    for ny, steps in ((64, 40000), (128, 160000), (256, 640000)):
        p, phi, u, ps = C.poiseuille2d(ny=ny, rho_ratio=1000.0, W=ny / 16.0, g=1e-6 * (64.0 / ny) ** 2)
        sim = lib.LBM(p)
        sim.init_fields(phi, u, ps)
        sim.step(steps)
        ph, uu, _ = sim.fields()
        sim.close()
        ux = uu[0, 0, :, 0].astype(np.float64)
        ufd = fd_poiseuille(ph[0, :, 0].astype(np.float64), p)
        errs[ny] = float(np.sqrt(((ux - ufd) ** 2).sum() / (ufd ** 2).sum()))
    o1, o2 = (np.log2(errs[a] / errs[2 * a]) for a in (64, 128))
    report("poiseuille_gpu", e64=errs[64], e128=errs[128], e256=errs[256], order_64_128=o1, order_128_256=o2)
    assert errs[64] < 0.03
    assert 1.7 < np.log2(errs[64] / errs[256]) / 2 < 2.5 and 1.7 < o1 < 2.5
    assert errs[256] < 1.5e-3
