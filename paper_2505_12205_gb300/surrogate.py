"""Learned fast-forward of planar-jet sweeps.

The workload: D2Q9 planar jets (``lbm_cases.jet2d``: 512 x 2048 nodes, inlet
slot 32 cells wide on y = 0, convective outlet at the top, periodic in x,
rho* = 100, mu* = 10, Re = 200) for Weber numbers in [1, 10].  The solver
writes snapshots every K steps; the network sees them 4x coarse-grained
(phi, u, v on 128 x 512, plus the Weber number as a constant channel) and
predicts the coarse fields K steps later.

The solver is both the fallback and the judge.  A prediction is refined to
the solver grid (bilinear), its interface re-sharpened to the equilibrium
width, its phase field corrected towards the mass budget by a correction
localised on the interface, and the solver restarts
from it (equilibrium populations, p* = 0, which the solver re-equilibrates).
It is accepted when the interface-position error is at most
``interface_bound`` cells of the solver grid -- both the mean distance
between the predicted interface and the solver's (phi = 1/2; symmetric
difference area over interface length) and the largest displacement of the
intact jet length (from the inlet to the first phi <= 1/2 over the nozzle
columns, the quantity behind a breakup length) -- and the mass error at most
``mass_bound``.

``fast_forward`` runs a case with the network in the loop: a window of K
solver steps checks the network's prediction of that window (the judge, at
the cost of one inference), and after a passing check the next ``skip``
windows are skipped by the network (prediction + restart each); after a
failing check the solver continues on its own.  Its result is compared with the solver alone
over the same span.

Everything on the path runs in the library's kernels (the solver through
include/lbm.h, the network and the field transfers through include/lbm_nn.h);
PyTorch provides device buffers and streams.
"""
from __future__ import annotations

import time

import numpy as np

import lbm_cases as C

from . import lbm, nn

FACTOR = 4            # coarse-graining of the solver grid
K = 200               # solver steps per prediction
U_SCALE = 20.0        # velocities are scaled to O(1) for the network (u_j = 0.05)
CIN = 8               # input channels: phi, u, v, Weber, zero padding
NOZZLE_HALF = 16      # half width of the inlet slot (lbm_cases.jet2d)
U_MAX = 0.15          # speed limit of a restart state (3 u_j)
# Width ratio of the phi = 1/2 interface profile after 4x box coarse-graining
# and bilinear refinement to that of the tanh profile of width W = 5 it came
# from (1.32 .. 1.39 over the sub-cell offsets of the interface); the restart
# re-sharpens the refined field by it (lbm_nn_sharpen).
SHARPEN = 1.35


def we_cond(We: float) -> float:
    return (We - 5.5) / 4.5


class Case:
    """One planar jet on the solver with device buffers for its fields."""

    def __init__(self, We, nx=512, ny=2048, stream=None):
        import torch
        self.torch = torch
        self.We = float(We)
        self.p, phi, u, ps = C.jet2d(nx=nx, ny=ny, We=We)
        self.nx, self.ny = nx, ny
        self.N = nx * ny
        self.stream = stream
        self.sim = lbm.LBM(self.p, stream=stream)
        self.sim.init_fields(phi, u, ps)
        self.t = 0
        dev = dict(dtype=torch.float32, device="cuda")
        self.phi = torch.zeros(self.N, **dev)
        self.u = torch.zeros(2 * self.N, **dev)
        self.sums = torch.zeros(4, dtype=torch.float64, device="cuda")
        self.hc, self.wc = ny // FACTOR, nx // FACTOR

    def close(self):
        self.sim.close()

    def step(self, n):
        self.sim.step(n)
        self.t += n

    def read_fields(self):
        lbm.lbm_get_fields(self.sim._h, self.phi, self.u, None)

    def coarse(self, x=None, xf=None):
        """Coarse network input x (bf16 [m][CIN]) and fields xf (f32 [m][3]) of the current state."""
        self.read_fields()
        nn.call("lbm_nn_coarsen", nn._p(self.phi), nn._p(self.u[:self.N]), nn._p(self.u[self.N:]), self.ny, self.nx,
                FACTOR, U_SCALE, we_cond(self.We), nn._p(x), CIN, nn._p(xf), nn._s(self.stream))

    def restart_from(self, pred, mass_target):
        """Solver state from a coarse prediction pred (f32 [m][3]): refined,
        re-sharpened, mass-projected, equilibrium populations with p* = 0."""
        restart_fields(pred, self.hc, self.wc, mass_target, self.phi, self.u, self.sums, self.stream)
        lbm.lbm_init_fields(self.sim._h, self.phi, self.u, None, n=self.N, dim=2)

    def mass(self):
        return float(self.sim.diag()["sum_phi"])


def restart_fields(pred, hc, wc, mass_target, phi, u, sums, stream=None):
    """The solver-grid fields a restart starts from, given a coarse prediction
    pred (f32 [hc * wc][3]): bilinear refinement (phi clamped to [0, 1],
    speed limited to U_MAX), the interface re-sharpened to the equilibrium
    width, and phi projected onto mass_target by an interface-localised
    correction.  phi: [N], u: [2 N] device buffers; sums: 2 doubles of scratch."""
    n = phi.numel()
    nn.call("lbm_nn_refine", nn._p(pred), hc, wc, FACTOR, U_SCALE, U_MAX, nn._p(phi), nn._p(u[:n]),
            nn._p(u[n:]), nn._s(stream))
    nn.call("lbm_nn_sharpen", nn._p(phi), n, SHARPEN, nn._s(stream))
    nn.call("lbm_nn_mass_project", nn._p(phi), n, float(mass_target), nn._p(sums), nn._s(stream))


def interface_stats(phi_a, phi_b, ny, nx, out, stream=None):
    """(mean distance between the interfaces, sum phi_a, sum phi_b)."""
    nn.call("lbm_nn_interface_stats", nn._p(phi_a), nn._p(phi_b), ny, nx, nn._p(out), nn._s(stream))
    o = out.cpu().numpy()
    return float(o[0] / max(o[1], 1.0)), float(o[2]), float(o[3])


def front_error(phi_a, phi_b, ny, nx, iout, x0=None, x1=None, stream=None):
    """Difference of the intact jet lengths of a and b (cells from the inlet
    to the first phi <= 1/2, largest over the nozzle columns [x0, x1))."""
    x0 = nx // 2 - NOZZLE_HALF if x0 is None else x0
    x1 = nx // 2 + NOZZLE_HALF if x1 is None else x1
    nn.call("lbm_nn_jet_length", nn._p(phi_a), nn._p(phi_b), ny, nx, x0, x1, nn._p(iout), nn._s(stream))
    la, lb = (int(v) for v in iout.cpu().numpy()[:2])
    return abs(la - lb)


def generate(We_list, t0, t1, nx=512, ny=2048, stream=None):
    """Coarse snapshots every K steps from t0 to t1 for each Weber number:
    X (bf16 [n][m][CIN]) inputs, Y (f32 [n][m][3]) the coarse fields K steps
    later, and the case index of each pair.  The kernels write the snapshots
    straight into the preallocated pair arrays."""
    import torch
    per = (t1 - t0) // K
    m = (ny // FACTOR) * (nx // FACTOR)
    X = torch.zeros(len(We_list) * per, m, CIN, dtype=torch.bfloat16, device="cuda")
    Y = torch.zeros(len(We_list) * per, m, 3, dtype=torch.float32, device="cuda")
    cases = np.repeat(np.arange(len(We_list)), per)
    for ci, We in enumerate(We_list):
        c = Case(We, nx=nx, ny=ny, stream=stream)
        c.step(t0)
        base = ci * per
        for snap in range(per + 1):
            if snap:
                c.step(K)
            c.coarse(x=X[base + snap] if snap < per else None, xf=Y[base + snap - 1] if snap else None)
        c.close()
    return X, Y, cases


def train(net, X, Y, idx, epochs, accum=4, lr=1e-3, decay=0.7, seed=0, log=None, nx=512, ny=2048):
    """Adam over the pairs idx, `accum` samples of gradient per step, the
    learning rate multiplied by `decay` after each epoch."""
    r = np.random.Generator(np.random.PCG64(seed))
    H, W = ny // FACTOR, nx // FACTOR
    hist = []
    for ep in range(epochs):
        order = r.permutation(idx)
        tot = 0.0
        for j, i in enumerate(order):
            A = net.forward(X[i], 1, H, W, target=Y[i])
            net.backward(X[i], 1, H, W, zero_grad=(j % accum == 0))
            tot += float(A["loss"].item())
            if j % accum == accum - 1 or j == len(order) - 1:
                net.adam_step(lr=lr * decay ** ep)
        hist.append(tot / len(order))
        if log:
            log("epoch %d loss %.3e" % (ep, hist[-1]))
    return hist


def evaluate(net, X, Y, idx, nx=512, ny=2048):
    """Mean loss over the pairs idx and that of the persistence prediction
    (the input fields themselves, i.e. a zero head)."""
    H, W = ny // FACTOR, nx // FACTOR
    import torch
    zero = torch.zeros(H * W, net.head, dtype=torch.float32, device="cuda")
    acc = torch.zeros(1, dtype=torch.float32, device="cuda")
    loss = pers = 0.0
    for i in idx:
        A = net.forward(X[i], 1, H, W, target=Y[i])
        loss += float(A["loss"].item())
        acc.zero_()
        nn.call("lbm_nn_mse", nn._p(zero), net.head, nn._p(X[i]), CIN, nn._p(Y[i]), 3, H * W, None, None, 0,
                nn._p(acc), nn._s(net.stream))
        pers += float(acc.item())
    return loss / len(idx), pers / len(idx)


def solver_twin(We, t0, t1, ref_phi, mode, eps=1e-6, every=2, seed=0, nx=512, ny=2048, stream=None):
    """The solver alone from t0 to t1 under a controlled disturbance, compared
    at t1 with the undisturbed solver's phi (ref_phi):
      'perturb': every g population scaled by 1 + eps r (r uniform in [-1, 1],
                 seeded) at t0 -- how far the flow itself carries a
                 disturbance at the level of float32 rounding;
      'restart': every `every`-th window of K steps ends with a restart from
                 the solver's own coarse-grained state (refined, mass-projected,
                 equilibrium with p* = 0) -- what a perfect network would give
                 through the same restart.
    Returns (mean interface distance, jet-length change, mass error, restarts)."""
    import torch
    c = Case(We, nx=nx, ny=ny, stream=stream)
    c.step(t0)
    restarts = 0
    if mode == "perturb":
        Q = 9
        f = torch.empty(Q * c.N, dtype=torch.float32, device="cuda")
        g = torch.empty(Q * c.N, dtype=torch.float32, device="cuda")
        lbm.lbm_get_populations(c.sim._h, f, g)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(C.SEED + 50 + seed)
        r = torch.rand(Q * c.N, generator=gen, device="cuda", dtype=torch.float32).mul_(2.0).sub_(1.0)
        g.mul_(r.mul_(eps).add_(1.0))
        lbm.lbm_set_populations(c.sim._h, f, g)
        c.step(t1 - t0)
    elif mode == "restart":
        xf = torch.zeros(c.hc * c.wc, 3, dtype=torch.float32, device="cuda")
        w = 0
        while c.t + K <= t1:
            c.step(K)
            w += 1
            if w % every == 0 and c.t < t1:
                c.coarse(xf=xf)
                c.restart_from(xf, c.mass())
                restarts += 1
        if c.t < t1:
            c.step(t1 - c.t)
    else:
        raise ValueError(mode)
    c.read_fields()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    iout = torch.zeros(2, dtype=torch.int32, device="cuda")
    dist, sa, sb = interface_stats(c.phi, ref_phi, ny, nx, out, stream)
    front = front_error(c.phi, ref_phi, ny, nx, iout, stream=stream)
    c.close()
    return dist, front, abs(sa - sb) / max(abs(sb), 1e-30), restarts


def fast_forward(net, We, t0, t1, interface_bound=1.0, mass_bound=1e-4, skip=1, nx=512, ny=2048, stream=None,
                 twins=False, solve=1):
    """Run one case from t0 to t1 with the network in the loop (after a
    passing check, once at least `solve` solver windows have run since the
    last skip, the next `skip` windows are predicted, one by one, instead of
    solved), and the same case with the solver alone; returns the
    comparison.  Every restart from a prediction moves the state a little
    (the coarse-graining loses detail), so fewer skips per window keep the end
    state closer to the solver's."""
    import torch
    H, W = ny // FACTOR, nx // FACTOR
    m = H * W
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream() if stream is None else stream
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    iout = torch.zeros(2, dtype=torch.int32, device="cuda")

    # solver alone
    ref = Case(We, nx=nx, ny=ny, stream=stream)
    ref.step(t0)
    torch.cuda.synchronize()
    ev0.record(st)
    ref.step(t1 - t0)
    ev1.record(st)
    torch.cuda.synchronize()
    ms_solver = ev0.elapsed_time(ev1)
    ref.read_fields()

    # network in the loop
    ff = Case(We, nx=nx, ny=ny, stream=stream)
    ff.step(t0)
    x = torch.zeros(m, CIN, dtype=torch.bfloat16, device="cuda")
    xb = torch.zeros(m, CIN, dtype=torch.bfloat16, device="cuda")
    phi_pred = torch.zeros(ff.N, dtype=torch.float32, device="cuda")
    u_pred = torch.zeros(2 * ff.N, dtype=torch.float32, device="cuda")
    rate = None
    windows = dict(solver=0, skipped=0, checked_pass=0, checked_fail=0)
    errs = []
    trusted = 0
    since_skip = 0                  # solver windows since the last skip
    torch.cuda.synchronize()
    ev0.record(st)
    t_wall = time.perf_counter()
    # the mass of the current state, tracked on the host: measured after a
    # solver window, the projection target after a skipped one (a restart
    # sets sum phi to it), so a skipped window needs no device round trip
    m_cur = ff.mass()
    while ff.t + K <= t1:
        m0 = m_cur
        ff.coarse(x=x)
        A = net.forward(x, 1, H, W)
        if trusted:
            # skip this window: restart from the prediction, mass from the budget
            target = m0 + K * (rate or 0.0)
            ff.restart_from(A["pred"], target)
            m_cur = target
            ff.t += K
            windows["skipped"] += 1
            trusted -= 1
            since_skip = 0
            continue
        # solver window, which also judges the network's prediction of it: the
        # fields a restart from the prediction would start from, with the mass
        # a skip would take (the budget extrapolated from the previous solver
        # window; none before the first, which therefore cannot pass)
        ff.step(K)
        windows["solver"] += 1
        since_skip += 1
        m1 = ff.mass()
        m_cur = m1
        target = m1 if rate is None else m0 + K * rate
        restart_fields(A["pred"], H, W, target, phi_pred, u_pred, out, stream)
        ff.read_fields()
        dist, sa, sb = interface_stats(phi_pred, ff.phi, ff.ny, ff.nx, out, stream)
        front = front_error(phi_pred, ff.phi, ff.ny, ff.nx, iout, stream)
        merr = abs(sa - sb) / max(abs(sb), 1e-30) if rate is not None else float("inf")
        rate = (m1 - m0) / K
        ok = dist <= interface_bound and front <= interface_bound and merr <= mass_bound
        errs.append((dist, front, merr))
        windows["checked_pass" if ok else "checked_fail"] += 1
        trusted = skip if (ok and since_skip >= solve) else 0
    ev1.record(st)
    torch.cuda.synchronize()
    ms_ff = ev0.elapsed_time(ev1)
    ff.read_fields()
    dist_end, sa, sb = interface_stats(ff.phi, ref.phi, ff.ny, ff.nx, out, stream)
    front_end = front_error(ff.phi, ref.phi, ff.ny, ff.nx, iout, stream)
    res = dict(We=We, t0=t0, t1=t1, ms_solver=ms_solver, ms_fast_forward=ms_ff,
               speedup=ms_solver / ms_ff, final_interface_distance=dist_end, final_front_error=front_end,
               final_mass_error=abs(sa - sb) / max(abs(sb), 1e-30), windows=windows,
               accepted_at_end=bool(dist_end <= interface_bound and front_end <= interface_bound
                                    and abs(sa - sb) / max(abs(sb), 1e-30) <= mass_bound),
               judged=[dict(interface=d, front=f, mass=e if np.isfinite(e) else None) for d, f, e in errs])
    if twins:
        for mode in ("perturb", "restart"):
            d, f, e, n = solver_twin(We, t0, t1, ref.phi, mode, every=skip + 1, nx=nx, ny=ny, stream=stream)
            res["twin_" + mode] = dict(final_interface_distance=d, final_front_error=f, final_mass_error=e,
                                       restarts=n)
    ref.close()
    ff.close()
    return res
