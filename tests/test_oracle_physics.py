"""Physics pins of the FP64 oracle on whole grids: closed forms and invariants
the paper and the mathematics fix.

  * uniform states are fixed points of the step (equilibria, streaming,
    periodic faces, inlet and outlet rules of App. B);
  * sum phi is conserved to round-off with periodic and bounce-back faces
    (eq:conservative_form; the paper's mass drift band is +-2e-6);
  * the centred drop keeps the grid's mirror and rotation symmetries;
  * a single-phase shear wave decays at nu k^2 with nu = tau c_s^2
    (eq:kinematic_viscosity);
  * a flat interface keeps the tanh profile of eq:kernel_function;
  * a 2D drop obeys Laplace's law dp = sigma / R (eq:laplace_law);
  * layered two-phase Poiseuille flow matches a finite-difference solution of
    eq:momentum_equation with the same smoothed rho(y), mu(y) (Sec. 5.3);
  (the open-face rules of App. B are pinned in test_oracle_faces.py).
"""
import numpy as np
import pytest

import lbm_cases as C


def run(oracle_mod, case, steps):
    p, phi, u, ps = case
    o = oracle_mod.Oracle(p)
    o.init_fields(phi, u, ps)
    o.step(steps)
    return o


@pytest.mark.parametrize("lat,shape", [(0, (1, 6, 7)), (1, (5, 4, 6))])
def test_uniform_flow_fixed_point_periodic(oracle_mod, lat, shape):
    case = C.uniform_flow(lat, shape)
    o = oracle_mod.Oracle(case[0])
    o.init_fields(*case[1:])
    f0, g0 = o.populations()
    o.step(20)
    f1, g1 = o.populations()
    assert np.abs(f1 - f0).max() < 1e-14 and np.abs(g1 - g0).max() < 1e-14
    phi, u, p = o.fields()
    assert np.allclose(phi, 0.7, atol=1e-15)
    for d in range(o.D):
        assert np.allclose(u[d], case[2][d], atol=1e-15)


@pytest.mark.parametrize("lat,shape", [(0, (1, 12, 5)), (1, (10, 4, 5))])
def test_uniform_plug_through_inlet_and_outlet(oracle_mod, lat, shape):
    """A uniform plug with phi = 1 entering through a nozzle wider than the face
    and leaving through the convective outlet is a fixed point."""
    D = 2 if lat == 0 else 3
    bc = [0, 0, 2, 3, 0, 0] if lat == 0 else [0, 0, 0, 0, 2, 3]
    uj = float(np.float32(0.03))       # the float32 field and the inlet speed agree
    uvec = [0.0, 0.0, 0.0]
    uvec[D - 1] = uj
    case = C.uniform_flow(lat, shape, u=uvec, phi=1.0, pstar=0.0, bc=bc, inlet_u=uj,
                          inlet_center=[2.0, 2.0], inlet_radius=1e6, W=4.0)
    o = oracle_mod.Oracle(case[0])
    o.init_fields(*case[1:])
    f0, g0 = o.populations()
    o.step(15)
    f1, g1 = o.populations()
    assert np.abs(f1 - f0).max() < 1e-14 and np.abs(g1 - g0).max() < 1e-14


@pytest.mark.parametrize("name", ["drop2d", "rt2d_walls", "drop3d"])
def test_sum_phi_conserved(oracle_mod, name):
    if name == "drop2d":
        case, steps = C.drop2d(n=40, R=10), 200
    elif name == "rt2d_walls":
        case, steps = C.rayleigh_taylor2d(L=32), 300
    else:
        case, steps = C.drop3d(n=14, R=4.0), 60
    p, phi, u, ps = case
    o = oracle_mod.Oracle(p)
    o.init_fields(phi, u, ps)
    s0 = o.fields()[0].sum()
    o.step(steps)
    phi1, u1, _ = o.fields()
    assert np.isfinite(phi1).all()
    assert abs(phi1.sum() - s0) / s0 < 1e-12


def test_drop2d_symmetries(oracle_mod):
    o = run(oracle_mod, C.drop2d(n=40, R=10), 150)
    phi, u, p = (a[0] if a.ndim == 3 else a[:, 0] for a in o.fields())
    scale = np.abs(u).max()
    assert scale > 0
    # mirror x -> n-1-x, y -> n-1-y and transpose (90 degree symmetry)
    assert np.abs(phi - phi[:, ::-1]).max() < 1e-13
    assert np.abs(phi - phi[::-1, :]).max() < 1e-13
    assert np.abs(phi - phi.T).max() < 1e-13
    assert np.abs(u[0] + u[0][:, ::-1]).max() < 1e-9 * scale
    assert np.abs(u[0] - u[0][::-1, :]).max() < 1e-9 * scale
    assert np.abs(u[0] - u[1].T).max() < 1e-9 * scale
    assert np.abs(p - p.T).max() < 1e-9 * np.abs(p).max()


def test_drop3d_symmetries(oracle_mod):
    o = run(oracle_mod, C.drop3d(n=14, R=4.0), 40)
    phi, u, p = o.fields()
    scale = np.abs(u).max()
    assert scale > 0
    for perm in [(0, 2, 1), (1, 0, 2), (2, 1, 0)]:
        assert np.abs(phi - phi.transpose(perm)).max() < 1e-13
    assert np.abs(phi - phi[:, :, ::-1]).max() < 1e-13
    # u_x(z,y,x) = u_y(z,x,y) under the x<->y swap, u_x odd in x
    assert np.abs(u[0] - u[1].transpose(0, 2, 1)).max() < 1e-9 * scale
    assert np.abs(u[0] + u[0][:, :, ::-1]).max() < 1e-9 * scale


@pytest.mark.parametrize("lat,axis_u,axis_k", [(0, 0, 1), (0, 1, 0), (1, 0, 2), (1, 2, 1)])
@pytest.mark.parametrize("tau", [0.1, 0.3, 1.5])
def test_shear_wave_decay_rate(oracle_mod, lat, axis_u, axis_k, tau):
    """u = U sin(k x) decays as exp(-nu k^2 t) with nu = tau c_s^2; the lattice
    correction is second order in k dx (4x smaller at twice the resolution)."""
    errs = []
    for n in (32, 64):
        p, phi, u, ps = C.shear_wave(lat, n=n, U=1e-4, tau=tau, axis_u=axis_u, axis_k=axis_k)
        o = oracle_mod.Oracle(p)
        o.init_fields(phi, u, ps)
        mode = u[axis_u] / 1e-4

        def amp():
            return (o.fields()[1][axis_u] * mode).sum() / (mode * mode).sum()
        o.step(100)            # let the non-equilibrium stress build up
        a1 = amp()
        o.step(300)
        a2 = amp()
        k = 2 * np.pi / n
        errs.append(-np.log(a2 / a1) / 300 / (tau / 3.0 * k * k) - 1.0)
    assert abs(errs[1]) < 4e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_flat_interface_keeps_tanh_profile(oracle_mod):
    W = 5.0
    p, phi, u, ps = C.flat_interface2d(nx=3, ny=80, W=W, sigma=1e-3)
    o = oracle_mod.Oracle(p)
    o.init_fields(phi, u, ps)
    o.step(3000)
    ph = o.fields()[0][0, :, 1]
    y = np.arange(80.0)
    # least-squares fit of the width of the lower interface around y = 20
    sel = (y > 5) & (y < 35)
    best = min(((np.square(ph[sel] - C.tanh_profile(y[sel] - y0, Wt)).sum(), Wt, y0)
                for Wt in np.linspace(4.5, 5.5, 101) for y0 in np.linspace(19.5, 20.5, 41)))
    assert abs(best[1] / W - 1) < 0.02
    assert abs(best[2] - 20.0) < 0.05
    assert np.abs(o.fields()[1]).max() < 1e-7


def laplace_dp(p_field, phi, R):
    n = phi.shape[-1]
    c = (n - 1) / 2.0
    yy, xx = np.mgrid[0:n, 0:n]
    r = np.hypot(xx - c, yy - c)
    return p_field[r < R - 6].mean() - p_field[r > R + 6].mean()


@pytest.mark.slow
def test_laplace_law_2d(oracle_mod):
    R, sigma = 16.0, 1e-3
    o = run(oracle_mod, C.drop2d(n=64, R=R, sigma=sigma, W=4.0, tau_H=0.5), 3000)
    phi, u, p = o.fields()
    dp = laplace_dp(p[0], phi[0], R)
    assert abs(dp / (sigma / R) - 1.0) < 0.03


def fd_poiseuille(phi, p):
    """Second-order FD solution of d/dy(mu du/dy) + rho g = 0 on nodes y_j = j,
    u = 0 on halfway walls at y = -1/2 and y = ny - 1/2, with the LBM's own
    mu(phi), rho(phi) (eq:momentum_equation)."""
    ph = np.clip(phi, 0, 1)
    rho = p["rho_L"] + ph * (p["rho_H"] - p["rho_L"])
    muL, muH = p["rho_L"] * p["tau_L"] / 3, p["rho_H"] * p["tau_H"] / 3
    mu = muL + ph * (muH - muL)
    n = len(phi)
    A = np.zeros((n, n))
    b = -rho * p["force"][0]
    for j in range(n):
        mm = 0.5 * (mu[j] + mu[j - 1]) if j > 0 else mu[0]
        mp = 0.5 * (mu[j] + mu[j + 1]) if j < n - 1 else mu[n - 1]
        # wall ghosts: u(-1) = -u(0), u(n) = -u(n-1)
        A[j, j] -= mm + mp
        if j > 0:
            A[j, j - 1] += mm
        else:
            A[j, j] -= mm
        if j < n - 1:
            A[j, j + 1] += mp
        else:
            A[j, j] -= mp
    return np.linalg.solve(A, b)


def poiseuille_error(oracle_mod, ny, rho_ratio, steps):
    W = ny / 16.0
    p, phi, u, ps = C.poiseuille2d(ny=ny, rho_ratio=rho_ratio, W=W, g=1e-6 * (64.0 / ny) ** 2)
    o = oracle_mod.Oracle(p)
    o.init_fields(phi, u, ps)
    o.step(steps)
    ph, uu, _ = o.fields()
    ux = uu[0, 0, :, 0]
    ufd = fd_poiseuille(ph[0, :, 0], p)
    return np.sqrt(((ux - ufd) ** 2).sum() / (ufd ** 2).sum())     # eq:l2_norm_error


@pytest.mark.slow
def test_poiseuille_two_phase_vs_fd_and_order():
    """rho* = 10 and 1000, mu* = 100 (Sec. 5.3).  At 64 nodes the LBM is within a
    few per cent of the FD solution; refining to 128 nodes (W scaled with the
    grid) cuts the error about 4x: second order, as the paper's slope -1.94."""
    from oracle import oracle as oracle_mod
    assert poiseuille_error(oracle_mod, 64, 10.0, 40000) < 1e-2
    e64 = poiseuille_error(oracle_mod, 64, 1000.0, 40000)
    e128 = poiseuille_error(oracle_mod, 128, 1000.0, 120000)
    assert e64 < 0.03
    order = np.log2(e64 / e128)
    assert 1.7 < order < 2.3


@pytest.mark.slow
def test_shear_flow_interface_returns_and_conserves_mass(oracle_mod, report):
    """Circular interface in a reversing shear flow (Sec. 5.3), phase field
    alone in the prescribed velocity, L0 = 100: sum phi is conserved to
    round-off and the interface returns close to its start.  (The paper
    prints a relative error of 8.58e-3 at L0 = 200; the readings of its time
    factor give 1.4e-2 to 4.4e-2 there, see the design notes.)"""
    import lbm_cases as C
    p, phi0, U, Tf = C.shear_flow_interface(L0=100)
    o = oracle_mod.Oracle(p)
    o.init_fields(phi0, None, None)
    T = 2 * Tf
    for t in range(T):
        o.advect(U, np.cos(np.pi * t / T), 1)
    phi = o.fields()[0].astype(np.float64)
    p0 = phi0.astype(np.float64)
    err = np.sqrt(((phi - p0) ** 2).sum() / (p0 ** 2).sum())
    mass = phi.sum() / p0.sum() - 1.0
    report("oracle_shear_flow_L100", err=err, mass=mass)
    assert abs(mass) < 1e-10
    assert err < 0.08
    # half way the interface is strongly deformed: far from the start
    o2 = oracle_mod.Oracle(p)
    o2.init_fields(phi0, None, None)
    for t in range(Tf):
        o2.advect(U, np.cos(np.pi * t / T), 1)
    mid = o2.fields()[0].astype(np.float64)
    assert np.sqrt(((mid - p0) ** 2).sum() / (p0 ** 2).sum()) > 0.5


@pytest.mark.parametrize("lat,shape,u", [(0, (1, 12, 9), (0.0, 0.03, 0.0)), (1, (7, 6, 5), (0.0, 0.02, 0.01))])
def test_free_slip_keeps_a_tangential_uniform_flow(oracle_mod, lat, shape, u):
    """Free slip (eq:free_slip_f/g) reflects specularly: a uniform flow along
    slip faces is a fixed point, while the same flow along no-slip walls is
    slowed at the walls."""
    p, phi, uu, ps = C.uniform_flow(lattice=lat, shape=shape, u=u)
    p["bc"] = [4, 4, 0, 0, 0, 0]
    o = oracle_mod.Oracle(p)
    o.init_fields(phi, uu, ps)
    o.step(50)
    ph, uo, _ = o.fields()
    assert np.abs(ph - phi).max() == 0.0
    assert np.abs(uo - uu).max() < 1e-14
    p["bc"] = [1, 1, 0, 0, 0, 0]
    o = oracle_mod.Oracle(p)
    o.init_fields(phi, uu, ps)
    o.step(50)
    assert np.abs(o.fields()[1] - uu).max() > 1e-3
