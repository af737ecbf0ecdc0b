"""Pins of the oracle's lattice constants, transformation matrices and
single-node collision against what the paper and the mathematics fix.

Lattices: eq:d3q19_velocities, eq:weights (D3Q19); D2Q9 ordering from the
momentum rows of eq:A1.  Matrices: eq:A1, eq:A2 (App. A).  Relaxation
matrix: eq:23 (D3Q19) and its D2Q9 analogue.  Collision: eq:mrt_collision,
eq:lbe_interface and the moment identities of the equilibria and forcing
terms.
"""
import itertools
import sys
import os

import numpy as np
import pytest

import lbm_cases as C

CS2 = 1.0 / 3.0
LATS = [(0, 9, 2), (1, 19, 3)]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "wmrt_matrices.txt")


def golden_matrices():
    mats, cur = {}, None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            mats[cur] = []
            continue
        mats[cur].append([int(v) for v in line.split()])
    return {k: np.array(v, float) for k, v in mats.items()}


@pytest.mark.parametrize("lat,Q,D", LATS)
def test_lattice_isotropy(oracle_mod, lat, Q, D):
    e, w, opp = oracle_mod.lattice(lat)
    assert e.shape == (Q, 3)
    assert np.all(e[:, D:] == 0)
    # distinct velocities, opposite table is an involution with e_opp = -e
    assert len({tuple(v) for v in e}) == Q
    assert np.all(e[opp] == -e) and np.all(opp[opp] == np.arange(Q))
    ed = e[:, :D].astype(float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(w @ ed, 0, atol=1e-16)
    assert np.allclose(np.einsum("a,ai,aj->ij", w, ed, ed), CS2 * np.eye(D), atol=1e-15)
    assert np.allclose(np.einsum("a,ai,aj,ak->ijk", w, ed, ed, ed), 0, atol=1e-16)
    t4 = np.einsum("a,ai,aj,ak,al->ijkl", w, ed, ed, ed, ed)
    d = np.eye(D)
    iso = CS2 ** 2 * (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
                      + np.einsum("il,jk->ijkl", d, d))
    assert np.allclose(t4, iso, atol=1e-15)
    # eq:weights: 12/36, 2/36, 1/36 in D3Q19 by speed class
    if lat == 1:
        speeds = (ed ** 2).sum(1)
        assert np.allclose(w[speeds == 0], 12 / 36) and np.allclose(w[speeds == 1], 2 / 36)
        assert np.allclose(w[speeds == 2], 1 / 36)
        assert (speeds == 1).sum() == 6 and (speeds == 2).sum() == 12


def test_matrices_match_printed(oracle_mod):
    g = golden_matrices()
    assert np.array_equal(oracle_mod.matrix(0), g["eq:A1"])
    assert np.array_equal(oracle_mod.matrix(1), g["eq:A2"])


@pytest.mark.parametrize("lat,Q,D", LATS)
def test_matrix_orthogonality(oracle_mod, lat, Q, D):
    M = oracle_mod.matrix(lat)
    e, w, _ = oracle_mod.lattice(lat)
    assert np.all(M[0] == 1)
    for d in range(D):
        assert np.array_equal(M[1 + d if lat == 1 else 3 + 2 * d], e[:, d])
    G = M @ M.T if lat == 0 else M @ np.diag(w) @ M.T
    assert np.allclose(G - np.diag(np.diag(G)), 0, atol=1e-14)
    assert np.all(np.diag(G) > 0)


@pytest.mark.parametrize("lat,Q,D", LATS)
@pytest.mark.parametrize("s", [0.3, 1.0, 1.25, 1.96])
def test_collision_matrix_eigenmodes(oracle_mod, lat, Q, D, s):
    """The deviatoric stress modes relax at s_nu; mass, momentum and the trace
    (bulk) mode at 1 (eq:23 and its D2Q9 analogue)."""
    Cm = oracle_mod.collision_matrix(lat, s)
    e, w, _ = oracle_mod.lattice(lat)
    ed = e[:, :D].astype(float)
    for i, j in itertools.combinations(range(D), 2):
        v = w * ed[:, i] * ed[:, j]
        assert np.allclose(Cm @ v, s * v, atol=1e-14)
        v = w * (ed[:, i] ** 2 - ed[:, j] ** 2)
        assert np.allclose(Cm @ v, s * v, atol=1e-14)
    for v in [w] + [w * ed[:, d] for d in range(D)] + [w * ((ed ** 2).sum(1) - D * CS2)]:
        assert np.allclose(Cm @ v, v, atol=1e-14)
    n_shear = D * (D + 1) // 2 - 1
    assert abs(np.trace(Cm) - (Q - n_shear * (1 - s))) < 1e-12
    if s == 1.0:
        assert np.allclose(Cm, np.eye(Q), atol=1e-14)


@pytest.mark.parametrize("lat,Q,D", LATS)
def test_moment_space_equals_distribution_space(oracle_mod, lat, Q, D):
    """Brute force on random cells: relaxing moments m = M f in moment space
    and transforming back gives the dense M^-1 S M used in velocity space."""
    M = golden_matrices()["eq:A1" if lat == 0 else "eq:A2"]
    shear = [7, 8] if lat == 0 else [4, 5, 6, 7, 8]
    r = C.rng(11)
    for _ in range(200):
        s = r.uniform(0.05, 1.99)
        x = r.standard_normal(Q)
        m = M @ x
        m[shear] *= s
        y = np.linalg.solve(M, m)
        assert np.allclose(oracle_mod.collision_matrix(lat, s) @ x, y, atol=1e-12)


def _node_ctx(oracle_mod, lat, **kw):
    p = C.base_params(lat, 1, 1, 1, **kw)
    return oracle_mod.Oracle(p)


def _equilibria(e, w, phi, u, pstar):
    eu = e @ u
    G = w * (1 + eu / CS2 + eu ** 2 / (2 * CS2 ** 2) - (u @ u) / (2 * CS2))
    return pstar * w + G - w, phi * G


@pytest.mark.parametrize("lat,Q,D", LATS)
def test_uniform_equilibrium_is_fixed_point(oracle_mod, lat, Q, D):
    e, w, _ = oracle_mod.lattice(lat)
    o = _node_ctx(oracle_mod, lat, rho_L=0.01, tau_L=0.9, tau_H=0.2, sigma=1e-3)
    r = C.rng(12)
    for _ in range(20):
        u = np.zeros(3)
        u[:D] = r.uniform(-0.05, 0.05, D)
        phi = r.uniform(0.0, 1.0)
        f, g = _equilibria(e, w, phi, u, r.uniform(-1e-3, 1e-3))
        fs, gs, out, t = o.collide_node(f, g, np.full(Q, phi))
        assert np.allclose(fs, f, atol=1e-16) and np.allclose(gs, g, atol=1e-16)
        assert np.allclose(out[1:1 + D], u[:D], atol=1e-16)


@pytest.mark.parametrize("lat,Q,D", LATS)
def test_collision_conservation_and_force(oracle_mod, lat, Q, D):
    """sum g* = sum g = phi, sum f* = sum f = p*, sum f* e = sum f e + F / rho
    (first moment of eq:force_term), for random non-equilibrium cells."""
    e, w, _ = oracle_mod.lattice(lat)
    o = _node_ctx(oracle_mod, lat, rho_L=0.01, tau_L=0.9, tau_H=0.2, sigma=1e-3,
                  force=[1e-5, -2e-5, 3e-5], rho_ref=0.01)
    r = C.rng(13)
    ed = e.astype(float)
    for _ in range(50):
        f = (r.random(Q) - 0.5) * 0.02 / Q
        g = r.random(Q) / Q
        phin = np.clip(g.sum() + 0.2 * (r.random(Q) - 0.5), -0.05, 1.05)
        phin[0] = g.sum()
        fs, gs, out, t = o.collide_node(f, g, phin)
        assert abs(gs.sum() - g.sum()) < 1e-15
        assert abs(fs.sum() - f.sum()) < 1e-15
        F = np.array([t["Fx"], t["Fy"], t["Fz"]])
        assert np.allclose(fs @ ed, f @ ed + F / t["rho"], atol=1e-14)
        # eq:velocity_update
        assert np.allclose(out[1:4], f @ ed + F / (2 * t["rho"]), atol=1e-15)


@pytest.mark.parametrize("lat,Q,D", LATS)
def test_stencils_exact_on_quadratics(oracle_mod, lat, Q, D):
    """eq:gradient_phi and eq:laplacian_phi are exact for quadratic phi."""
    e, w, _ = oracle_mod.lattice(lat)
    o = _node_ctx(oracle_mod, lat)
    r = C.rng(14)
    for _ in range(10):
        a0, b, H = r.random(), r.standard_normal(3), r.standard_normal((3, 3))
        H = H + H.T
        b[D:] = 0
        H[D:, :] = 0
        H[:, D:] = 0
        phin = np.array([a0 + b @ v + 0.5 * v @ H @ v for v in e.astype(float)])
        g = np.zeros(Q)
        g[0] = a0
        _, _, _, t = o.collide_node(np.zeros(Q), g, phin)
        assert np.allclose([t["gx"], t["gy"], t["gz"]], b, atol=1e-13)
        assert abs(t["lap"] - np.trace(H)) < 1e-13


@pytest.mark.parametrize("W", [4.0, 5.0, 8.0])
def test_chemical_potential_vanishes_on_tanh_profile(oracle_mod, W):
    """With beta = 12 sigma / W and kappa = 3 sigma W / 2 (eq:beta_kappa_relation)
    the tanh profile of eq:kernel_function is an equilibrium: mu_phi ~ 0 up to
    the O(1/W^2) error of the discrete Laplacian, far below either of its two
    terms.  The sign printed in eq:chemical_potential would double the terms."""
    e, w, _ = oracle_mod.lattice(0)
    sigma = 1e-3
    o = _node_ctx(oracle_mod, 0, sigma=sigma, W=W)
    beta = 12 * sigma / W
    worst = 0.0
    for z0 in np.linspace(-W, W, 21):
        phin = C.tanh_profile(z0 + e[:, 0], W)
        g = np.zeros(9)
        g[0] = phin[0]
        _, _, _, t = o.collide_node(np.zeros(9), g, phin)
        worst = max(worst, abs(t["mu_phi"]) / (beta / 8))
    # discrete residual ~ 2.5 / W^2 of the double-well scale beta/8; the
    # printed sign would leave about 3 of it
    assert worst * W * W < 3.0


def test_prosperetti_reference_curve_limits():
    """The repaired Prosperetti curve starts at 1; for small viscosity it
    oscillates at omega_0 = sqrt(sigma k^3 / (rho_H + rho_L)), and its damping
    is set by the interfacial boundary layer, so it grows like sqrt(nu)."""
    pytest.importorskip("scipy")
    from prosperetti import amplitude
    k, sigma = 2 * np.pi / 256, 1e-2
    om0 = np.sqrt(sigma * k ** 3 / 2.0)
    assert abs(amplitude([0.0], k, 1e-3, sigma, 1.0, 1.0)[0] - 1.0) < 1e-9
    t = np.linspace(0, 4 * 2 * np.pi / om0, 8001)

    def crossings_and_decay(nu):
        eta = amplitude(t, k, nu, sigma, 1.0, 1.0)
        zc = [t[i] - eta[i] * (t[i + 1] - t[i]) / (eta[i + 1] - eta[i])
              for i in range(len(t) - 1) if eta[i] * eta[i + 1] < 0]
        env = np.abs(eta)
        peaks = [i for i in range(1, len(t) - 1) if env[i] >= env[i - 1] and env[i] > env[i + 1]]
        rate = -np.log(env[peaks[-1]] / env[peaks[0]]) / (t[peaks[-1]] - t[peaks[0]])
        return np.array(zc), rate
    zc, r1 = crossings_and_decay(1e-6)
    assert abs(2 * np.mean(np.diff(zc)) * om0 / (2 * np.pi) - 1) < 5e-3
    _, r4 = crossings_and_decay(4e-6)
    assert 1.6 < r4 / r1 < 2.4
