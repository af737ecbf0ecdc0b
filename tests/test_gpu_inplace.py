"""The in-place (AA) layout against the A/B layout, through the C ABI.

With layout 1 a context holds one copy of each population set and its steps
alternate between writing each node's post-collision populations into its
own opposite slots and reading/writing them at the neighbours.  The
arithmetic per node is the same as with two copies, so every state -- after
even and odd step counts, with every face type, float32 and float16 storage,
from equilibrium fields or from a restored checkpoint -- must equal the A/B
context's bit for bit, and the population memory must halve.
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


CASES = {
    # name: (lattice, shape (nz, ny, nx), bc)
    "d2q9_periodic": (0, (1, 23, 70), [0, 0, 0, 0, 0, 0]),
    "d2q9_walls": (0, (1, 17, 19), [1, 1, 1, 1, 0, 0]),
    "d2q9_jet": (0, (1, 29, 67), [0, 0, 2, 3, 0, 0]),
    "d2q9_freeslip_jet": (0, (1, 29, 67), [4, 4, 2, 3, 0, 0]),
    "d3q19_periodic": (1, (9, 7, 37), [0] * 6),
    "d3q19_walls": (1, (11, 9, 13), [1, 1, 0, 0, 1, 1]),
    "d3q19_jet": (1, (12, 10, 35), [0, 0, 1, 1, 2, 3]),
    "d3q19_freeslip": (1, (9, 11, 13), [4, 4, 4, 4, 1, 1]),
    "d3q19_freeslip_jet": (1, (12, 10, 33), [4, 4, 4, 4, 2, 3]),
}


def _params(name, storage=0, scheme=0):
    lat, (nz, ny, nx), bc = CASES[name]
    p = C.base_params(lat, nx, ny, nz, rho_L=0.05, tau_L=0.3, tau_H=0.1, sigma=2e-3, W=4.0,
                      force=[1e-5, -2e-5, 3e-5], rho_ref=0.05, inlet_u=0.04,
                      inlet_center=[nx / 2.0 - 0.3, ny / 2.0 + 0.2], inlet_radius=3.5)
    p["bc"] = bc
    p["storage"] = storage
    p["outlet_scheme"] = scheme
    return p


def _same(a, b):
    fa, ga = a.populations()
    fb, gb = b.populations()
    return np.array_equal(fa, fb) and np.array_equal(ga, gb)


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_inplace_equals_ab_bitwise(lib, name, storage):
    p = _params(name, storage)
    f, g = C.random_state(p, seed_offset=sum(name.encode()) % 997)
    f, g = f.astype(np.float32), g.astype(np.float32)
    ab = lib.LBM(p)
    aa = lib.LBM(dict(p, layout=1))
    ab.set_populations(f, g)
    aa.set_populations(f, g)
    for n in (1, 2, 17, 16, 3):              # both parities, single launches and graph replays
        ab.step(n)
        aa.step(n)
        assert _same(ab, aa), (name, storage, n)
    for x, y in zip(ab.fields(), aa.fields()):
        assert np.array_equal(x, y)
    da, db = ab.diag(), aa.diag()
    for k in ("sum_phi", "sum_p_in", "sum_p_out", "max_speed", "n_in", "n_out", "finite"):
        assert da[k] == db[k], k


@pytest.mark.parametrize("scheme", [1, 2])
def test_inplace_outlet_speed_schemes(lib, scheme):
    """U_max and U_ave outlet speeds (a reduction over the outlet layer read
    through the layout) on the small 3D jet from equilibrium fields."""
    p, phi, u, ps = C.jet3d(nx=24, ny=24, nz=48, Rn=4.0)
    p = dict(p, outlet_scheme=scheme, bc=[4, 4, 4, 4, 2, 3])
    ab, aa = lib.LBM(p), lib.LBM(dict(p, layout=1))
    ab.init_fields(phi, u, ps)
    aa.init_fields(phi, u, ps)
    ab.step(41)
    aa.step(41)
    assert _same(ab, aa)


def test_inplace_checkpoint_crosses_layouts(lib):
    """A checkpoint taken from the in-place context after an odd step count
    (swapped state) restores into an A/B context and the other way round."""
    p, phi, u, ps = C.jet2d(nx=64, ny=96, half_width=6.0, W=4.0, stub=10.0)
    aa = lib.LBM(dict(p, layout=1))
    aa.init_fields(phi, u, ps)
    aa.step(23)
    f, g = aa.populations()
    ab = lib.LBM(p)
    ab.set_populations(f, g)
    aa.step(30)
    ab.step(30)
    assert _same(ab, aa)
    f, g = ab.populations()
    aa2 = lib.LBM(dict(p, layout=1))
    aa2.set_populations(f, g)
    aa2.step(5)
    ab.step(5)
    assert _same(ab, aa2)


def test_inplace_in_step_diagnostics_and_advection(lib):
    p, phi, u, ps = C.drop2d(n=40, R=10.0)
    p = dict(p, layout=1, diag_every=5)
    sim = lib.LBM(p)
    sim.init_fields(phi, u, ps)
    sim.step(12)
    rec, step = sim.diag_last()
    assert step == 10 and rec["finite"] == 1
    with pytest.raises(lib.LbmError) as e:
        sim.advect(np.zeros((2, 1, 40, 40), np.float32), 1.0, 1)
    assert e.value.code == lib.LBM_ERR_ARG


def test_inplace_halves_population_memory(lib):
    import torch
    p = C.base_params(1, 256, 256, 64)            # 4.2 M nodes: 0.64 GB per copy of both sets
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ab = lib.LBM(p)
    used_ab = free0 - torch.cuda.mem_get_info()[0]
    ab.close()
    free1 = torch.cuda.mem_get_info()[0]
    aa = lib.LBM(dict(p, layout=1))
    used_aa = free1 - torch.cuda.mem_get_info()[0]
    aa.close()
    state = 2 * 19 * 4 * 256 * 256 * 64
    assert used_ab >= 2 * state
    assert used_aa < 0.62 * used_ab, (used_aa, used_ab)
