"""Parity at the full sizes the bench times, in the launch configuration it
times: the 3D jet (D3Q19, 256 x 256 x 1024, inlet and outlet) and the tiled
2D Rayleigh-Taylor workload (D2Q9, 8192 x 32768, walls).

The GPU takes one step of the whole grid from a seeded random state drawn on
the device; sampled nodes (interior, next to the inlet, outlet and walls) are
compared with the oracle's step of the patch around each (patch_step.py),
at the one-step tolerances of test_gpu_parity.
"""
import numpy as np
import pytest

import lbm_cases as C
import patch_step as PS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_12205_gb300 import build, lbm
    build.build()
    lbm.load()
    from oracle import oracle
    oracle.build()
    return torch, lbm, oracle


def close(a, b, l2=1e-5, mx=5e-5):
    a = np.asarray(a, np.float64)
    scale = np.abs(b).max()
    return (np.linalg.norm(a - b) <= l2 * np.linalg.norm(b) + 1e-30
            and np.abs(a - b).max() <= mx * scale + 1e-30)


def run(torch, lbm, orc, p, seed, samples, report, tag):
    f0, g0 = C.random_state_device(p, seed_offset=seed)
    sim = lbm.LBM(p, stream=torch.cuda.current_stream())
    sim.set_populations(f0.reshape(-1), g0.reshape(-1))
    sim.step(1)
    f1, g1 = torch.empty_like(f0), torch.empty_like(g0)
    lbm.lbm_get_populations(sim._h, f1.reshape(-1), g1.reshape(-1))
    torch.cuda.synchronize()
    sim.close()

    def get_patch(idx):
        zz, yy, xx = (torch.as_tensor(v, device=f0.device) for v in idx)
        take = lambda a: a.index_select(1, zz).index_select(2, yy).index_select(3, xx).double().cpu().numpy()
        return take(f0), take(g0)

    worst = 0.0
    for (z, y, x, kind) in samples:
        rf, rg = PS.node_step(orc, p, z, y, x, kind, get_patch)
        gf = f1[:, z, y, x].double().cpu().numpy()
        gg = g1[:, z, y, x].double().cpu().numpy()
        worst = max(worst, np.abs(gf - rf).max() / np.abs(rf).max(), np.abs(gg - rg).max() / np.abs(rg).max())
        assert close(gg, rg), (z, y, x, kind, np.abs(gg - rg).max())
        assert close(gf, rf), (z, y, x, kind, np.abs(gf - rf).max())
    report(tag, samples=len(samples), worst_rel_max=worst)


def test_jet3d_full_size_sampled_nodes(env, report):
    torch, lbm, orc = env
    p, _, _, _ = C.jet3d()
    run(torch, lbm, orc, p, 101, PS.samples_jet(p, C.rng(102)), report, "fullsize_jet3d_256x256x1024")


def test_rt2d_tiled_full_size_sampled_nodes(env, report):
    torch, lbm, orc = env
    p, _, _, _ = C.rayleigh_taylor2d(L=256, periods=32, height=32768)
    run(torch, lbm, orc, p, 103, PS.samples_walls2d(p, C.rng(104)), report, "fullsize_rt2d_8192x32768")
