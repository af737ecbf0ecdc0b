"""Seeded synthetic inputs shared by the CUDA library's tests, the benchmark
and the FP64 oracle.

This module only builds *inputs*: case parameters and initial macroscopic
fields (phi, u, p*) in float32, plus seeded random population states for
single-step checks.  It holds none of the lattice Boltzmann arithmetic (no
equilibria, no collision, no streaming); each implementation derives its own
populations from these fields.

Field layout: ``[nz][ny][nx]`` with x fastest; the velocity is ``D``
consecutive planes.  Parameters are a plain dict whose keys mirror the C
parameter struct (visc_model 0: mu linear in phi, 1: tau linear in phi) (``lattice, nx, ny, nz, bc[6], visc_model, rho_L, rho_H,
tau_L, tau_H, sigma, W, mobility, force[3], rho_ref, inlet_u,
inlet_center[2], inlet_radius``, optionally ``outlet_scheme`` 0/1/2 for the
local / maximum / average outlet speed).

Case recipes follow the paper's validation and application sections and the
workload sizes used by the benchmark:
  * stationary drop (Sec. 5.2): tanh drop of radius R, heavy inside, centred
    at ((nx-1)/2, (ny-1)/2), periodic box, zero velocity;
  * Rayleigh-Taylor (Sec. 5.5, table tab:rayleigh_spec case a): heavy fluid
    above light, interface y0 = ny/2 + 0.1 L cos(2 pi x / L), walls top and
    bottom, periodic in x, at rest with the hydrostatic pressure of the body
    force; U0 = sqrt(g L) = 0.04 sets g, the Reynolds, Peclet and capillary
    numbers set tau_H, M and sigma;
  * liquid jet (Sec. 6): circular plug inlet on the z = 0 face, convective
    outlet on the top z face, periodic sides, gravity along the jet;
  * two-phase Poiseuille (Sec. 5.3), flat interface, single-phase shear wave
    and capillary wave set-ups for the physics checks;
  * batched sweep: many drop and capillary-wave cases of random size and
    material parameters, advanced together.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 0x250512205

D2Q9, D3Q19 = 0, 1
PERIODIC, WALL, INLET, OUTFLOW, FREESLIP = 0, 1, 2, 3, 4


def rng(seed_offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED + seed_offset))


def tanh_profile(z, W):
    """eq:kernel_function with phi_L = 0, phi_H = 1: 1/2 + 1/2 tanh(2 z / W)."""
    return 0.5 + 0.5 * np.tanh(2.0 * np.asarray(z, np.float64) / W)


def base_params(lattice, nx, ny, nz=1, **kw):
    p = dict(lattice=lattice, nx=nx, ny=ny, nz=nz, bc=[PERIODIC] * 6, visc_model=0,
             rho_L=1e-3, rho_H=1.0, tau_L=0.5, tau_H=0.5, sigma=1e-4, W=5.0,
             mobility=0.02, force=[0.0, 0.0, 0.0], rho_ref=0.0, inlet_u=0.0,
             inlet_center=[0.0, 0.0], inlet_radius=0.0)
    p.update(kw)
    return p


def tau_L_from_ratios(tau_H, rho_ratio, mu_ratio):
    """tau_L such that mu_H / mu_L = mu_ratio with nu = tau c_s^2."""
    return tau_H * rho_ratio / mu_ratio


def _zeros_u(D, shape):
    return np.zeros((D,) + shape, np.float32)


# --------------------------------------------------------------- 2D drop

def drop2d(n=128, R=25.0, rho_ratio=1000.0, mu_ratio=100.0, sigma=1e-4, W=5.0,
           mobility=0.02, tau_H=0.8):
    """Stationary 2D drop, D2Q9, periodic box (the 128 x 128, R = 25 case)."""
    p = base_params(D2Q9, n, n, 1, rho_H=1.0, rho_L=1.0 / rho_ratio, tau_H=tau_H,
                    tau_L=tau_L_from_ratios(tau_H, rho_ratio, mu_ratio), sigma=sigma,
                    W=W, mobility=mobility)
    y, x = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64),
                       indexing="ij")
    c = (n - 1) / 2.0
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2)
    phi = tanh_profile(R - r, W).astype(np.float32)[None]
    return p, phi, _zeros_u(2, (1, n, n)), None


def drop3d(n=32, R=8.0, rho_ratio=1000.0, mu_ratio=100.0, sigma=1e-3, W=4.0,
           mobility=0.02, tau_H=0.5):
    """Stationary 3D drop, D3Q19, periodic box (Sec. 5.2, Laplace law 2 sigma / R)."""
    p = base_params(D3Q19, n, n, n, rho_H=1.0, rho_L=1.0 / rho_ratio, tau_H=tau_H,
                    tau_L=tau_L_from_ratios(tau_H, rho_ratio, mu_ratio), sigma=sigma,
                    W=W, mobility=mobility)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    c = (n - 1) / 2.0
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    phi = tanh_profile(R - r, W).astype(np.float32)
    return p, phi, _zeros_u(3, (n, n, n)), None


# -------------------------------------------------------- Rayleigh-Taylor

def rayleigh_taylor2d(L=256, height=None, W=5.0, At=0.5, Re=3000.0, Pe=1000.0,
                      Ca=0.26, U0=0.04, mu_ratio=1.0, periods=1):
    """2D Rayleigh-Taylor instability, D2Q9, L x 4L, walls top/bottom, periodic x.

    periods > 1 repeats the same physics (the parameters of wavelength L)
    periods times along x, on a domain periods*L wide and `height` high: the
    throughput workload of the HBM roofline (8192 x 32768 = 32 x 32 copies of
    the 256 x 1024 case's area)."""
    ny = 4 * L if height is None else height
    rho_H = 1.0
    rho_L = rho_H * (1.0 - At) / (1.0 + At)
    g = U0 * U0 / L
    mu_H = rho_H * U0 * L / Re
    tau_H = mu_H / (rho_H / 3.0)
    mu_L = mu_H / mu_ratio
    tau_L = mu_L / (rho_L / 3.0)
    nx = L * periods
    p = base_params(D2Q9, nx, ny, 1, rho_H=rho_H, rho_L=rho_L, tau_H=tau_H, tau_L=tau_L,
                    sigma=mu_H * U0 / Ca, W=W, mobility=U0 * L / Pe,
                    force=[0.0, -g, 0.0], rho_ref=rho_L)
    p["bc"] = [PERIODIC, PERIODIC, WALL, WALL, PERIODIC, PERIODIC]
    x = np.arange(nx, dtype=np.float64)
    y0 = ny / 2.0 + 0.1 * L * np.cos(2.0 * np.pi * x / L)
    phi = np.empty((1, ny, nx), np.float32)                  # heavy on top
    pstar = np.empty((1, ny, nx), np.float32)
    drho = rho_H - rho_L
    # Fluid at rest in hydrostatic balance with the body force
    # F_b = (rho - rho_L) g: p(y) = p(y + 1) + (F_b(y) + F_b(y + 1)) / 2 down
    # from the top row (trapezoid rule), p* = p / (rho c_s^2); row blocks from
    # the top carry the running sum.  The level is set by p = 0 at mid-height
    # of column 0 (near the interface, where p* enters the pressure force).
    f0 = tanh_profile(np.arange(ny, dtype=np.float64) - y0[0], W) * drho * g
    p_mid = (0.5 * (f0[:-1] + f0[1:]))[ny // 2:].sum()
    carry = np.full(nx, -p_mid)
    fb_above = None
    for r1 in range(ny, 0, -1024):                           # row blocks: bounded temporaries
        r0 = max(0, r1 - 1024)
        y = np.arange(r0, r1, dtype=np.float64)[:, None]
        ph = tanh_profile(y - y0[None, :], W)
        phi[0, r0:r1] = ph
        fb = ph * drho * g                                   # |F_b| (downwards)
        half = 0.5 * (fb[:-1] + fb[1:])                      # between rows y and y + 1
        step = np.concatenate([half, (0.5 * (fb[-1] + fb_above))[None] if fb_above is not None
                               else np.zeros((1, nx))])
        pr = carry[None, :] + np.cumsum(step[::-1], axis=0)[::-1]
        carry = pr[0].copy()
        fb_above = fb[0].copy()
        pstar[0, r0:r1] = pr / ((rho_L + ph * drho) / 3.0)
    return p, phi, _zeros_u(2, (1, ny, nx)), pstar


# -------------------------------------------------------------- 3D jet

def jet3d(nx=256, ny=256, nz=1024, Rn=16.0, We=2.2, Re=200.0, u_j=0.05,
          rho_ratio=100.0, mu_ratio=10.0, W=5.0, mobility=0.02, Bo=0.0658,
          stub=None):
    """Liquid jet into quiescent gas, D3Q19: plug inlet of radius Rn on z = 0,
    convective outlet on z = nz-1, periodic sides, gravity along +z.

    Re = rho_H u_j D / mu_H and We = rho_H u_j^2 D / sigma fix mu_H and sigma;
    g follows from the Bond number Bo = rho_H g D^2 / sigma.  The initial field
    is a liquid stub of length ``stub`` (default D) above the nozzle in gas at
    rest.
    """
    D = 2.0 * Rn
    rho_H, rho_L = 1.0, 1.0 / rho_ratio
    mu_H = rho_H * u_j * D / Re
    tau_H = mu_H / (rho_H / 3.0)
    tau_L = tau_L_from_ratios(tau_H, rho_ratio, mu_ratio)
    sigma = rho_H * u_j * u_j * D / We
    g = Bo * sigma / (rho_H * D * D)
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    p = base_params(D3Q19, nx, ny, nz, rho_H=rho_H, rho_L=rho_L, tau_H=tau_H,
                    tau_L=tau_L, sigma=sigma, W=W, mobility=mobility,
                    force=[0.0, 0.0, g], rho_ref=rho_L, inlet_u=u_j,
                    inlet_center=[cx, cy], inlet_radius=Rn)
    p["bc"] = [PERIODIC, PERIODIC, PERIODIC, PERIODIC, INLET, OUTFLOW]
    stub = D if stub is None else stub
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    z = np.arange(nz, dtype=np.float64)
    r = np.sqrt((x[None, :] - cx) ** 2 + (y[:, None] - cy) ** 2)      # [ny][nx]
    radial = tanh_profile(Rn - r, W)
    axial = tanh_profile(stub - z, W)                                  # [nz]
    phi = (axial[:, None, None] * radial[None, :, :]).astype(np.float32)
    return p, phi, _zeros_u(3, (nz, ny, nx)), None


def jet2d(nx=512, ny=2048, half_width=16.0, We=5.0, Re=200.0, u_j=0.05,
          rho_ratio=100.0, mu_ratio=10.0, W=5.0, mobility=0.02, Bo=0.0,
          stub=None):
    """Planar jet, D2Q9: plug inlet slot |x - xc| < half_width on the y = 0
    face, convective outlet on y = ny-1, periodic in x (the planar-jet shape
    of the learned fast-forward workload)."""
    D = 2.0 * half_width
    rho_H, rho_L = 1.0, 1.0 / rho_ratio
    mu_H = rho_H * u_j * D / Re
    tau_H = mu_H / (rho_H / 3.0)
    tau_L = tau_L_from_ratios(tau_H, rho_ratio, mu_ratio)
    sigma = rho_H * u_j * u_j * D / We
    g = Bo * sigma / (rho_H * D * D)
    cx = (nx - 1) / 2.0
    p = base_params(D2Q9, nx, ny, 1, rho_H=rho_H, rho_L=rho_L, tau_H=tau_H,
                    tau_L=tau_L, sigma=sigma, W=W, mobility=mobility,
                    force=[0.0, g, 0.0], rho_ref=rho_L, inlet_u=u_j,
                    inlet_center=[cx, 0.0], inlet_radius=half_width)
    p["bc"] = [PERIODIC, PERIODIC, INLET, OUTFLOW, PERIODIC, PERIODIC]
    stub = D if stub is None else stub
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    radial = tanh_profile(half_width - np.abs(x - cx), W)
    axial = tanh_profile(stub - y, W)
    phi = (axial[:, None] * radial[None, :]).astype(np.float32)[None]
    return p, phi, _zeros_u(2, (1, ny, nx)), None


def uniform_flow(lattice=D2Q9, shape=(1, 8, 8), u=(0.02, -0.01, 0.015), phi=0.7,
                 pstar=1e-3, bc=None, **kw):
    """Uniform state: constant phi, u, p* (no gradients, no body force)."""
    nz, ny, nx = shape
    D = 2 if lattice == D2Q9 else 3
    p = base_params(lattice, nx, ny, nz, **kw)
    if bc is not None:
        p["bc"] = list(bc)
    uu = np.zeros((D,) + shape, np.float32)
    for d in range(D):
        uu[d] = u[d]
    return p, np.full(shape, phi, np.float32), uu, np.full(shape, pstar, np.float32)


# ----------------------------------------------------- physics-check cases

def flat_interface2d(nx=4, ny=64, W=5.0, sigma=1e-3, rho_ratio=10.0, tau=0.5,
                     mobility=0.02):
    """Two flat interfaces (periodic in y), heavy band in the middle, at rest."""
    p = base_params(D2Q9, nx, ny, 1, rho_H=1.0, rho_L=1.0 / rho_ratio, tau_H=tau,
                    tau_L=tau, sigma=sigma, W=W, mobility=mobility)
    y = np.arange(ny, dtype=np.float64)
    a, b = ny / 4.0, 3.0 * ny / 4.0
    phi1d = tanh_profile(y - a, W) + tanh_profile(b - y, W) - 1.0
    phi = np.broadcast_to(phi1d[:, None], (ny, nx)).astype(np.float32)[None].copy()
    return p, phi, _zeros_u(2, (1, ny, nx)), None


def poiseuille2d(ny=64, nx=2, rho_ratio=1000.0, mu_ratio=100.0, tau_H=0.5, W=4.0,
                 g=1e-6):
    """Layered two-phase Poiseuille flow (Sec. 5.3): light fluid in the lower
    half, heavy in the upper half, walls at y = -1/2 and y = ny - 1/2,
    body force rho g along x, mu linear in phi (eq:dynamic_viscosity)."""
    p = base_params(D2Q9, nx, ny, 1, rho_H=1.0, rho_L=1.0 / rho_ratio, tau_H=tau_H,
                    tau_L=tau_L_from_ratios(tau_H, rho_ratio, mu_ratio), sigma=0.0,
                    W=W, mobility=0.02, force=[g, 0.0, 0.0], rho_ref=0.0, visc_model=0)
    p["bc"] = [PERIODIC, PERIODIC, WALL, WALL, PERIODIC, PERIODIC]
    y = np.arange(ny, dtype=np.float64)
    Lh = ny / 2.0 - 0.5          # interface half way between the walls
    phi1d = tanh_profile(y - Lh, W)
    phi = np.broadcast_to(phi1d[:, None], (ny, nx)).astype(np.float32)[None].copy()
    return p, phi, _zeros_u(2, (1, ny, nx)), None


def shear_wave(lattice=D2Q9, n=32, U=1e-3, tau=0.3, axis_u=0, axis_k=1):
    """Single-phase (phi = 1) decaying shear wave u_axis_u = U sin(2 pi k . x)."""
    dims = [4, 4, 1 if lattice == D2Q9 else 4]     # x, y, z
    dims[axis_k] = n
    shape3 = (dims[2], dims[1], dims[0])
    nz, ny, nx = shape3
    p = base_params(lattice, nx, ny, nz, rho_H=1.0, rho_L=1.0, tau_H=tau, tau_L=tau,
                    sigma=0.0, W=4.0, mobility=0.02)
    D = 2 if lattice == D2Q9 else 3
    coords = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xk = [coords[2], coords[1], coords[0]][axis_k].astype(np.float64)
    u = np.zeros((D,) + shape3, np.float32)
    u[axis_u] = (U * np.sin(2.0 * np.pi * xk / n)).astype(np.float32)
    phi = np.ones(shape3, np.float32)
    return p, phi, u, None


def capillary_wave2d(L=32, height=None, amp=None, sigma=1e-2, rho_ratio=1.0, nu=0.02,
                     W=4.0, mobility=0.02):
    """Capillary wave (Sec. 5.1): heavy fluid below, light above, interface
    y = H/2 + amp cos(2 pi x / L), equal kinematic viscosity in both phases,
    walls top and bottom, periodic x."""
    ny = 2 * L if height is None else height
    amp = 0.05 * L if amp is None else amp
    tau = nu * 3.0
    p = base_params(D2Q9, L, ny, 1, rho_H=1.0, rho_L=1.0 / rho_ratio, tau_H=tau,
                    tau_L=tau, sigma=sigma, W=W, mobility=mobility)
    p["bc"] = [PERIODIC, PERIODIC, WALL, WALL, PERIODIC, PERIODIC]
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(L, dtype=np.float64),
                       indexing="ij")
    y0 = ny / 2.0 + amp * np.cos(2.0 * np.pi * x / L)
    phi = tanh_profile(y0 - y, W).astype(np.float32)[None]       # heavy below
    return p, phi, _zeros_u(2, (1, ny, L)), None


# ---------------------------------------------------- batched sweep cases

def sweep_case(kind, L, rho_ratio, sigma, R=None, W=5.0, mobility=0.02, tau=0.5):
    """One case of a parameter sweep on an L x L D2Q9 grid with equal
    kinematic viscosity in both phases (tau_L = tau_H, tau linear in phi, so
    tau is the same everywhere):
      kind 0: stationary drop of radius R, centred, periodic box (Sec. 5.2);
      kind 1: capillary wave (Sec. 5.1), heavy fluid below, interface
              y = L/2 + 0.01 L cos(2 pi x / L), walls top and bottom,
              periodic x."""
    p = base_params(D2Q9, L, L, 1, rho_H=1.0, rho_L=1.0 / rho_ratio, tau_H=tau, tau_L=tau,
                    sigma=sigma, W=W, mobility=mobility, visc_model=1)
    y, x = np.meshgrid(np.arange(L, dtype=np.float64), np.arange(L, dtype=np.float64),
                       indexing="ij")
    if kind == 0:
        c = (L - 1) / 2.0
        phi = tanh_profile(R - np.sqrt((x - c) ** 2 + (y - c) ** 2), W)
    else:
        p["bc"] = [PERIODIC, PERIODIC, WALL, WALL, PERIODIC, PERIODIC]
        y0 = L / 2.0 + 0.01 * L * np.cos(2.0 * np.pi * x / L)
        phi = tanh_profile(y0 - y, W)
    return p, phi.astype(np.float32)[None], _zeros_u(2, (1, L, L)), None


def sweep_cases(n=512, L_min=64, L_max=512, seed_offset=4):
    """The seeded sweep of n cases: L ~ U{L_min..L_max}, kind ~ Bernoulli(1/2)
    (drop / capillary wave), drop radius R ~ U[8, 0.3 L], density ratio
    log-uniform in [10, 1000], sigma log-uniform in [1e-5, 1e-3]."""
    r = rng(seed_offset)
    out = []
    for _ in range(n):
        L = int(r.integers(L_min, L_max + 1))
        kind = int(r.integers(0, 2))
        R = float(r.uniform(8.0, max(8.0, 0.3 * L)))
        rho_ratio = float(np.exp(r.uniform(np.log(10.0), np.log(1000.0))))
        sigma = float(np.exp(r.uniform(np.log(1e-5), np.log(1e-3))))
        out.append(sweep_case(kind, L, rho_ratio, sigma, R=R))
    return out


# ------------------------------------------ circular interface in shear flow

def shear_flow_interface(L0=200, U0=0.04, mobility=0.0002, W=3.0, R=None, centre=(100.0, 60.0)):
    """Circular interface in a reversing shear flow (Sec. 5.3): periodic
    L0 x L0 box, circle of radius L0/5 centred at (100, 60) (scaled with L0),
    velocity U(x, y) cos(pi t / (2 T_f)), T_f = L0 / U0, with
    U = (U0 sin^2(pi x / L0) sin(2 pi y / L0), -U0 sin^2(pi y / L0) sin(2 pi x / L0)).
    Returns (params, phi0, U planes [2][1][L0][L0], T_f)."""
    R = L0 / 5.0 if R is None else R
    cx, cy = centre[0] * L0 / 200.0, centre[1] * L0 / 200.0
    p = base_params(D2Q9, L0, L0, 1, rho_L=1.0, rho_H=1.0, tau_L=0.5, tau_H=0.5, sigma=0.0, W=W,
                    mobility=mobility)
    y, x = np.meshgrid(np.arange(L0, dtype=np.float64), np.arange(L0, dtype=np.float64), indexing="ij")
    phi = tanh_profile(R - np.sqrt((x - cx) ** 2 + (y - cy) ** 2), W).astype(np.float32)[None]
    U = np.zeros((2, 1, L0, L0), np.float32)
    U[0, 0] = U0 * np.sin(np.pi * x / L0) ** 2 * np.sin(2 * np.pi * y / L0)
    U[1, 0] = -U0 * np.sin(np.pi * y / L0) ** 2 * np.sin(2 * np.pi * x / L0)
    return p, phi, U, int(round(L0 / U0))


# ------------------------------------------------- random states (1 step)

def random_state_device(params, seed_offset=0, du=0.02, dphi=0.6, device="cuda"):
    """The recipe of random_state drawn on the GPU (torch's seeded generator)
    for grids too large to build on the host: float32 tensors f, g of shape
    [Q][nz][ny][nx] on the device."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(SEED + seed_offset)
    lat = params["lattice"]
    Q = 9 if lat == D2Q9 else 19
    shape = (params.get("nz", 1), params["ny"], params["nx"])

    def rnd(*s):
        return torch.rand(*s, generator=gen, device=device, dtype=torch.float32)

    phi = 0.5 + dphi * (rnd(*shape) - 0.5)
    f = rnd(Q, *shape).sub_(0.5).mul_(du).add_(1e-3 * (rnd(*shape) - 0.5)).div_(Q)
    g = rnd(Q, *shape).sub_(0.5).mul_(du).add_(1.0).mul_(phi / Q)
    return f, g


def random_state(params, seed_offset=0, du=0.02, dphi=0.6):
    """Seeded random but physical-looking post-stream populations:
    returns (f, g) float64 arrays [Q][nz][ny][nx] built as smooth random
    fields plus small random perturbations per population (not equilibria)."""
    r = rng(seed_offset)
    lat = params["lattice"]
    Q = 9 if lat == D2Q9 else 19
    shape = (params.get("nz", 1), params["ny"], params["nx"])
    phi = 0.5 + dphi * (r.random(shape) - 0.5)
    f = ((r.random((Q,) + shape) - 0.5) * du + 1e-3 * (r.random(shape) - 0.5)) / Q
    g = phi[None] / Q * (1.0 + du * (r.random((Q,) + shape) - 0.5))
    return f.astype(np.float32).astype(np.float64), g.astype(np.float32).astype(np.float64)
