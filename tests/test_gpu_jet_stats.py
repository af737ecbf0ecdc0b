"""Jet post-processing on the GPU (lbm_jet_stats) against the reference
components (oracle/jet_oracle.py) on the same phase field: integer results
(components, breakup length, drop volumes) must agree exactly."""
import numpy as np
import pytest

import lbm_cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pytest.importorskip("scipy")
    from paper_2505_12205_gb300 import build, lbm
    build.build()
    lbm.load()
    return lbm


def check(lib, p, phi, dim, report, name):
    from oracle import jet_oracle as J
    sim = lib.LBM(p)
    sim.init_fields(phi, None, None)
    g = sim.jet_stats(0.5)
    field = sim.fields()[0]
    arr = field[0] if dim == 2 else field
    bc = p["bc"]
    periodic = (bc[2] == 0, bc[0] == 0) if dim == 2 else (bc[4] == 0, bc[2] == 0, bc[0] == 0)
    r = J.jet_stats(arr, 0.5, periodic, dim)
    report("jet_stats_" + name, n=g["n_components"], L_b=g["breakup_length"], d=g["mean_drop_diameter"])
    for k in ("n_components", "has_jet", "breakup_length", "n_drops", "drop_volume"):
        assert g[k] == r[k], (k, g[k], r[k])
    assert sorted(g["drop_volumes"].tolist()) == r["drop_volumes"]
    assert np.isclose(g["mean_drop_diameter"], r["mean_drop_diameter"])
    sim.close()
    return g


def test_synthetic_3d_components(lib, report):
    nz, ny, nx = 40, 20, 24
    phi = np.full((nz, ny, nx), 0.1, np.float32)
    phi[0:15, 8:12, 10:14] = 0.9
    phi[20:23, 5:8, 3:6] = 0.9
    phi[30:32, 14:16, 0:2] = 0.9
    phi[30:32, 14:16, 22:24] = 0.9
    phi[35, 2, 2] = 0.9
    p = C.base_params(1, nx, ny, nz, rho_L=0.1)
    p["bc"] = [0, 0, 0, 0, 1, 1]
    g = check(lib, p, phi, 3, report, "synthetic3d")
    assert g["n_components"] == 4 and g["breakup_length"] == 15.0
    p["bc"] = [0, 0, 1, 1, 1, 1]                 # y no longer periodic: nothing changes here
    check(lib, p, phi, 3, report, "synthetic3d_walls")


def test_synthetic_2d_components(lib, report):
    ny, nx = 64, 48
    phi = np.full((1, ny, nx), 0.1, np.float32)
    phi[0, 0:20, 20:28] = 0.9
    phi[0, 30:34, 0:3] = 0.9
    phi[0, 30:34, 45:48] = 0.9                   # wraps across x
    phi[0, 50:53, 10:12] = 0.9
    phi[0, 60, 5] = phi[0, 61, 6] = 0.9          # diagonal contact: two drops
    p = C.base_params(0, nx, ny, 1, rho_L=0.1)
    p["bc"] = [0, 0, 1, 1, 0, 0]
    g = check(lib, p, phi, 2, report, "synthetic2d")
    assert g["n_components"] == 5 and g["breakup_length"] == 20.0


def test_jet_run_statistics_match_the_reference(lib, report):
    """A small 3D jet after 1500 steps, with the paper's free-slip sides."""
    p, phi, u, ps = C.jet3d(nx=32, ny=32, nz=96, Rn=4.0, We=1.0)
    p["bc"] = [4, 4, 4, 4, 2, 3]
    sim = lib.LBM(p)
    sim.init_fields(phi, u, ps)
    sim.step(1500)
    g = sim.jet_stats(0.5)
    field = sim.fields()[0]
    from oracle import jet_oracle as J
    r = J.jet_stats(field, 0.5, (False, False, False), 3)
    report("jet_stats_run", n=g["n_components"], L_b=g["breakup_length"], drops=g["n_drops"])
    for k in ("n_components", "has_jet", "breakup_length", "n_drops", "drop_volume"):
        assert g[k] == r[k], (k, g[k], r[k])
    assert g["has_jet"] == 1 and g["breakup_length"] > 0
