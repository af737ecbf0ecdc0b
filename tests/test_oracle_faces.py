"""Pins of the oracle's open-face rules (App. B) on hand-built states.

Inlet (eq:velocity_boundary_u, eq:velocity_boundary_distribution,
eq:mass_conservation): the velocity rule acts on f' = f + F/2
(eq:force_term).  At an inlet node the forces that need derivatives of phi
are not evaluated, so F is the body force F_b = (rho(phi_in) - rho_ref) g of
eq:gravity_force.  After the rule, at every inlet node,
    sum_a f'_a e_a = u_in    and    sum_a g_a = phi_in.
Since sum_a (F_a / 2) e_a = F / (2 rho) on an isotropic lattice
(sum_a w_a e_a e_a = c_s^2 I), the first condition reads
sum_a f_a e_a + F_b / (2 rho) = u_in.  The cases carry a body force with
both normal and tangential components, so a rule that drops the shift fails.

Outlet (eq:implicit_convective, eq:convective_f/g): on a single column the
rule is checked against a worked example computed by hand: populations of
layer N at time t (the old state) all 2 (f) and 1/2 (g); after streaming,
layer N-1 holds f = 3 except the population along +n, and g = 1/10.  The
outlet speed U is the first moment of f along n at layer N-1; lambda = U
clamped to [0, 1]; chi(N) = (chi_old(N) + lambda chi(N-1)) / (1 + lambda).
"""
import numpy as np
import pytest

import lbm_cases as C


# ------------------------------------------------------------------ inlet

@pytest.mark.parametrize("lat,shape", [(0, (1, 24, 30)), (1, (16, 12, 12))])
def test_inlet_rule_on_shifted_populations(oracle_mod, lat, shape):
    nz, ny, nx = shape
    if lat == 0:
        case = C.jet2d(nx=nx, ny=ny, half_width=5.0, W=4.0, stub=6.0)
    else:
        case = C.jet3d(nx=nx, ny=ny, nz=nz, Rn=3.0, W=4.0, stub=5.0)
    p = dict(case[0])
    p["force"] = [2e-4, 3e-4, -1e-4] if lat == 1 else [2e-4, -3e-4, 0.0]
    o = oracle_mod.Oracle(p)
    o.init_fields(*case[1:])
    e, w, _ = oracle_mod.lattice(lat)
    D = 2 if lat == 0 else 3
    L = D - 1
    if lat == 0:
        r = np.abs(np.arange(nx) - p["inlet_center"][0])
    else:
        yy, xx = np.mgrid[0:ny, 0:nx]
        r = np.hypot(xx - p["inlet_center"][0], yy - p["inlet_center"][1]).reshape(-1)
    phi_in = C.tanh_profile(p["inlet_radius"] - r, p["W"])
    u_in = np.zeros((D, r.size))
    u_in[L] = np.where(r < p["inlet_radius"], p["inlet_u"], 0.0)
    rho = p["rho_L"] + np.clip(phi_in, 0.0, 1.0) * (p["rho_H"] - p["rho_L"])
    Fb = np.array(p["force"][:D])[:, None] * (rho - p["rho_ref"])[None, :]
    for _ in range(3):
        o.step(5)
        f, g = o.populations()
        if lat == 0:
            fi, gi = f[:, 0, 0, :], g[:, 0, 0, :]                # [Q][x]
        else:
            fi, gi = f[:, 0, :, :].reshape(19, -1), g[:, 0, :, :].reshape(19, -1)
        j = np.einsum("ad,an->dn", e[:, :D].astype(float), fi)
        assert np.abs(gi.sum(0) - phi_in).max() < 1e-14
        # sum f' e = sum f e + F / (2 rho) = u_in
        assert np.abs(j + Fb / (2.0 * rho) - u_in).max() < 1e-14
        # the shift is visible: without it the rule would give sum f e = u_in
        assert np.abs(j - u_in).max() > 1e-5
        # and the macroscopic update finds u_in at the inlet nodes
        uf = o.fields()[1]
        ui = uf[:, 0, 0, :] if lat == 0 else uf[:, 0].reshape(D, -1)
        assert np.abs(ui - u_in).max() < 1e-12


# ----------------------------------------------------------------- outlet

def _column_case(oracle_mod, lat, scheme):
    """A grid whose outlet layer has one column per value of U in
    (0.25, -0.3, 1.7) (2D) or (0.25, 1.7) (3D); returns the oracle, the
    index of the population along +n and the populations after the rule."""
    if lat == 0:
        p = C.base_params(0, 3, 4, 1)
        p["bc"] = [0, 0, 1, 3, 0, 0]                 # wall below, outlet on top
        shape, cols = (1, 4, 3), [(0, None, 0), (1, None, 1), (2, None, 2)]
    else:
        p = C.base_params(1, 2, 1, 4)
        p["bc"] = [0, 0, 0, 0, 1, 3]
        shape, cols = (4, 1, 2), [(0, 0, 0), (1, 0, 2)]
    p["outlet_scheme"] = scheme
    o = oracle_mod.Oracle(p)
    e, _, _ = oracle_mod.lattice(lat)
    D = 2 if lat == 0 else 3
    L = D - 1
    n_up = [0, 0, 0]
    n_up[L] = 1
    up = [a for a in range(o.Q) if list(e[a]) == n_up][0]
    fA = np.full((o.Q,) + shape, 2.0)
    gA = np.full((o.Q,) + shape, 0.5)
    o.set_populations(fA, gA)
    fB = np.full((o.Q,) + shape, 3.0)
    gB = np.full((o.Q,) + shape, 0.1)
    extra = [0.25, -0.3, 1.7]                        # f_up - 3 = U at layer N-1
    for (x, y, k) in cols:
        idx = (up, 0, 2, x) if lat == 0 else (up, 2, 0, x)
        fB[idx] = 3.0 + extra[k]
    fo, go = o.apply_faces(fB, gB)
    return o, up, fB, gB, fo, go, cols


def _layer(a, lat, x):
    """populations of the outlet node of column x: [Q]"""
    return a[:, 0, 3, x] if lat == 0 else a[:, 3, 0, x]


@pytest.mark.parametrize("lat", [0, 1])
def test_outlet_single_column_local_speed(oracle_mod, lat):
    o, up, fB, gB, fo, go, cols = _column_case(oracle_mod, lat, 0)
    # hand-computed: U = 0.25 -> lambda = 1/4: f = (2 + 3/4) / (5/4) = 2.2,
    # f_up = (2 + 3.25/4) / (5/4) = 2.25, g = (1/2 + 1/40) / (5/4) = 0.42;
    # U = -0.3 -> lambda = 0: f = 2, g = 1/2 (the old layer, exactly);
    # U = 1.7 -> lambda = 1: f = 5/2, f_up = 3.35, g = 3/10
    want = {0: (2.2, 2.25, 0.42), 1: (2.0, 2.0, 0.5), 2: (2.5, 3.35, 0.3)}
    for (x, _, k) in cols:
        f, g = _layer(fo, lat, x), _layer(go, lat, x)
        wf, wup, wg = want[k]
        others = [a for a in range(o.Q) if a != up]
        assert np.abs(f[others] - wf).max() < 1e-14, (k, f)
        assert abs(f[up] - wup) < 1e-14, (k, f[up])
        assert np.abs(g - wg).max() < 1e-14, (k, g)
    # the other layers are not touched
    below = (slice(None), slice(None), slice(0, 3)) if lat == 0 else (slice(None), slice(0, 3))
    assert np.array_equal(fo[below], fB[below]) and np.array_equal(go[below], gB[below])


@pytest.mark.parametrize("scheme", [1, 2])
def test_outlet_max_and_average_speed(oracle_mod, scheme):
    """eq:velocity_options on the 2D column case: U_max = 1.7 -> lambda = 1 on
    every column; U_ave = (0.25 - 0.3 + 1.7) / 3 = 0.55 -> lambda = 0.55."""
    o, up, fB, gB, fo, go, cols = _column_case(oracle_mod, 0, scheme)
    fup = {0: 3.25, 1: 2.7, 2: 4.7}
    for (x, _, k) in cols:
        f, g = _layer(fo, 0, x), _layer(go, 0, x)
        if scheme == 1:
            # lambda = 1: the mean of the old and new layers
            wf, wup, wg = 2.5, {0: 2.625, 1: 2.35, 2: 3.35}[k], 0.3
        else:
            # lambda = 0.55: f = (2 + 1.65) / 1.55, g = (0.5 + 0.055) / 1.55
            wf, wup, wg = 3.65 / 1.55, (2.0 + 0.55 * fup[k]) / 1.55, 0.555 / 1.55
        others = [a for a in range(o.Q) if a != up]
        assert np.abs(f[others] - wf).max() < 1e-14
        assert abs(f[up] - wup) < 1e-14
        assert np.abs(g - wg).max() < 1e-14


def test_inlet_needs_an_opposite_outlet(oracle_mod):
    """An inlet without the convective outlet opposite is rejected."""
    p = C.jet2d(nx=16, ny=16, half_width=3.0, W=4.0)[0]
    assert oracle_mod.validate(p)
    p["bc"] = [0, 0, 2, 1, 0, 0]
    assert not oracle_mod.validate(p)
    p["bc"] = [0, 0, 2, 3, 0, 0]
    p["W"] = 1.5
    assert not oracle_mod.validate(p)
