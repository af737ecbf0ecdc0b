"""The patch method of the full-size parity tests (patch_step.py), pinned on
the CPU: the oracle's one-step result at sampled nodes of a small jet and a
small walled 2D case, computed from the patch around each node, equals the
oracle's own full-grid step at those nodes (to FP64 rounding).  A patch too
small for the step's reach, or a wrong face condition on the patch, fails."""
import numpy as np
import pytest

import lbm_cases as C
import patch_step as PS


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def full_step(orc, p, seed):
    f0, g0 = C.random_state(p, seed_offset=seed)
    o = orc.Oracle(p)
    o.set_populations(f0, g0)
    o.step(1)
    f1, g1 = o.populations()
    o.close()
    return f0, g0, f1, g1


def check(orc, p, f0, g0, f1, g1, samples, radius=PS.R):
    def get_patch(idx):
        zz, yy, xx = idx
        take = lambda a: a[:, zz][:, :, yy][:, :, :, xx]
        return take(f0), take(g0)
    worst = 0.0
    for (z, y, x, kind) in samples:
        rf, rg = PS.node_step(orc, p, z, y, x, kind, get_patch)
        worst = max(worst, np.abs(rf - f1[:, z, y, x]).max() / np.abs(f1[:, z, y, x]).max(),
                    np.abs(rg - g1[:, z, y, x]).max() / np.abs(g1[:, z, y, x]).max())
    return worst


def test_patches_reproduce_the_full_grid_step_jet(orc):
    p, _, _, _ = C.jet3d(nx=16, ny=16, nz=20, Rn=3.0)
    state = full_step(orc, p, 11)
    s = PS.samples_jet(p, C.rng(12), n_interior=12)
    assert check(orc, p, *state, s) < 1e-12


def test_patches_reproduce_the_full_grid_step_walls2d(orc):
    p, _, _, _ = C.rayleigh_taylor2d(L=32, periods=2, height=40)
    state = full_step(orc, p, 13)
    s = PS.samples_walls2d(p, C.rng(14), n_interior=12)
    assert check(orc, p, *state, s) < 1e-12


def test_a_patch_of_radius_one_is_too_small(orc, monkeypatch):
    """The step reaches two nodes: a radius-1 periodic patch wraps inside
    that reach and must disagree with the full grid."""
    p, _, _, _ = C.rayleigh_taylor2d(L=32, periods=2, height=40)
    state = full_step(orc, p, 15)
    monkeypatch.setattr(PS, "R", 1)
    s = [(0, 20, 10, "interior"), (0, 25, 40, "interior")]
    assert check(orc, p, *state, s) > 1e-9
