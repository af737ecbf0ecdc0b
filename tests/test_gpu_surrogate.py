"""The learned fast-forward's solver-side kernels and loop on a small planar
jet (128 x 512, 4x coarse 32 x 128): coarse-graining and refinement, the
interface-localised mass projection, the interface comparison, and one
train / evaluate / fast-forward round."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_12205_gb300 import build, nn, surrogate
    build.build()
    nn.load()
    return torch, nn, surrogate


def test_coarsen_refine_mass_and_interface_kernels(env):
    torch, nn, S = env
    ny, nx, f = 64, 48, 4
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    phi = (0.5 + 0.5 * np.tanh((20.0 - np.hypot(x - 24.0, y - 30.0)) / 2.5)).astype(np.float32)
    u = (0.01 * np.sin(2 * np.pi * x / nx)).astype(np.float32)
    v = np.full((ny, nx), 0.02, np.float32)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
    pd, ud, vd = d(phi), d(u), d(v)
    m = (ny // f) * (nx // f)
    xb = torch.zeros(m, 8, dtype=torch.bfloat16, device="cuda")
    xf = torch.zeros(m, 3, dtype=torch.float32, device="cuda")
    nn.call("lbm_nn_coarsen", nn._p(pd), nn._p(ud), nn._p(vd), ny, nx, f, 20.0, 0.3, nn._p(xb), 8, nn._p(xf), None)
    ref = phi.reshape(ny // f, f, nx // f, f).mean(axis=(1, 3))
    assert np.allclose(xf.cpu().numpy()[:, 0], ref.reshape(-1), atol=1e-6)
    assert np.allclose(xf.cpu().numpy()[:, 2], 0.4, atol=1e-6)                       # v * 20
    assert np.allclose(xb.float().cpu().numpy()[:, 3], 0.3, atol=2e-3)               # condition channel
    assert np.all(xb.float().cpu().numpy()[:, 4:] == 0)
    pf, uf, vf = (torch.zeros(ny * nx, dtype=torch.float32, device="cuda") for _ in range(3))
    nn.call("lbm_nn_refine", nn._p(xf), ny // f, nx // f, f, 20.0, 1.0, nn._p(pf), nn._p(uf), nn._p(vf), None)
    assert np.allclose(vf.cpu().numpy(), 0.02, atol=1e-7)                             # constants survive
    assert np.abs(pf.cpu().numpy() - phi.reshape(-1)).mean() < 0.05                   # smooth field, 4x coarse
    # re-sharpening: the formula of include/lbm_nn.h in float64, the phi = 1/2
    # level set kept, a coarse-grained and refined tanh profile brought back
    # to its width
    xs = np.linspace(-12.0, 12.0, 4001)
    prof = (0.5 + 0.5 * np.tanh(2.0 * xs / (5.0 * 1.35))).astype(np.float32)
    sd = d(prof)
    nn.call("lbm_nn_sharpen", nn._p(sd), prof.size, 1.35, None)
    q = np.clip(prof.astype(np.float64), 1e-6, 1 - 1e-6)
    ref_s = 0.5 + 0.5 * np.tanh(1.35 * np.arctanh(2 * q - 1))
    got_s = sd.cpu().numpy()
    assert np.abs(got_s - ref_s).max() < 2e-6
    assert np.abs(got_s - (0.5 + 0.5 * np.tanh(2.0 * xs / 5.0))).max() < 2e-6
    half = d(np.full(7, 0.5, np.float32))
    nn.call("lbm_nn_sharpen", nn._p(half), 7, 1.35, None)
    assert np.all(half.cpu().numpy() == 0.5)
    # mass projection onto the interface band
    sums = torch.zeros(2, dtype=torch.float64, device="cuda")
    target = float(phi.sum()) * 1.01
    nn.call("lbm_nn_mass_project", nn._p(pd), ny * nx, target, nn._p(sums), None)
    after = pd.cpu().numpy()
    assert abs(after.sum() / target - 1.0) < 1e-5
    assert np.all(after[phi.reshape(-1) < 1e-6] < 1e-5)                               # pure phases barely touched
    # interface distance: identical fields 0, a one-cell shift about 1
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    dist, _, _ = S.interface_stats(d(phi), d(phi), ny, nx, out)
    assert dist == 0.0
    dist, _, _ = S.interface_stats(d(np.roll(phi, 1, axis=1)), d(phi), ny, nx, out)
    assert 0.4 < dist < 1.2
    iout = torch.zeros(2, dtype=torch.int32, device="cuda")
    col = np.zeros((ny, nx), np.float32)
    col[:20, 20:28] = 1.0                                                             # a jet 20 cells long
    longer = col.copy()
    longer[20:23, 22:25] = 1.0                                                        # 3 cells longer
    assert S.front_error(d(col), d(col), ny, nx, iout, 16, 32) == 0
    assert S.front_error(d(longer), d(col), ny, nx, iout, 16, 32) == 3


def test_train_and_fast_forward_round_on_a_small_jet(env, report):
    torch, nn, S = env
    nx, ny, t0, t1 = 128, 512, 1000, 3000
    X, Y, cases = S.generate([2.0, 6.0], t0, t1, nx=nx, ny=ny)
    assert X.shape[0] == 2 * (t1 - t0) // S.K and bool(torch.isfinite(Y).all())
    net = S.nn.UNet(cin=S.CIN, ch=(16, 32, 32, 64))
    from oracle import nn_oracle
    net.set_params(nn_oracle.init_params(S.CIN, [16, 32, 32, 64], 8, seed=3))
    idx = np.arange(X.shape[0])
    hist = S.train(net, X, Y, idx, epochs=6, accum=2, lr=1e-3, nx=nx, ny=ny)
    loss, pers = S.evaluate(net, X, Y, idx, nx=nx, ny=ny)
    report("surrogate_small_train", first=hist[0], last=hist[-1], eval=loss, persistence=pers)
    assert hist[-1] < hist[0]
    res = S.fast_forward(net, 4.0, t0, t1, nx=nx, ny=ny)
    w = res["windows"]
    assert w["solver"] + w["skipped"] == (t1 - t0) // S.K
    assert w["checked_pass"] + w["checked_fail"] == w["solver"]
    assert np.isfinite(res["final_interface_distance"]) and res["ms_fast_forward"] > 0
    report("surrogate_small_ff", speedup=res["speedup"], final_dist=res["final_interface_distance"],
           final_mass=res["final_mass_error"], skipped=w["skipped"], solver=w["solver"])


def test_restart_from_a_coarse_grained_state_stays_finite(env, report):
    """The restart path without the network: a solver state coarse-grained
    4x, refined, mass-projected and restarted runs K steps and stays finite,
    close to the solver's own continuation."""
    torch, nn, S = env
    nx, ny = 128, 512
    c = S.Case(4.0, nx=nx, ny=ny)
    ref = S.Case(4.0, nx=nx, ny=ny)
    c.step(2000)
    ref.step(2000)
    m = c.hc * c.wc
    xf = torch.zeros(m, 3, dtype=torch.float32, device="cuda")
    c.coarse(xf=xf)
    m0 = c.mass()
    c.restart_from(xf, m0)
    assert abs(c.mass() / m0 - 1) < 1e-5
    c.step(S.K)
    ref.step(S.K)
    d = c.sim.diag()
    assert d["finite"] == 1
    c.read_fields()
    ref.read_fields()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    iout = torch.zeros(2, dtype=torch.int32, device="cuda")
    dist, _, _ = S.interface_stats(c.phi, ref.phi, ny, nx, out)
    front = S.front_error(c.phi, ref.phi, ny, nx, iout)
    report("surrogate_restart_persistence", dist=dist, front=front)
    assert dist < 3.0
    c.close()
    ref.close()


def test_solver_twins_on_a_small_jet(env, report):
    """The twins the fast-forward is measured against: an undisturbed twin
    (eps = 0) reproduces the solver's interface exactly, a 1e-6 disturbance and
    restarts from the solver's own coarse-grained state stay finite."""
    torch, nn, S = env
    nx, ny, t0, t1 = 128, 512, 1000, 1600
    ref = S.Case(4.0, nx=nx, ny=ny)
    ref.step(t1)
    ref.read_fields()
    d0, f0, m0, _ = S.solver_twin(4.0, t0, t1, ref.phi, "perturb", eps=0.0, nx=nx, ny=ny)
    assert d0 == 0.0 and f0 == 0 and m0 < 1e-12     # the mass sums are atomic (order varies)
    d1, f1, m1, _ = S.solver_twin(4.0, t0, t1, ref.phi, "perturb", eps=1e-6, nx=nx, ny=ny)
    d2, f2, m2, n2 = S.solver_twin(4.0, t0, t1, ref.phi, "restart", every=2, nx=nx, ny=ny)
    assert n2 == 1
    assert np.isfinite([d1, m1, d2, m2]).all() and d2 < 3.0
    report("surrogate_twins_small", perturbed=d1, restarted=d2, restarted_mass=m2)
    ref.close()
