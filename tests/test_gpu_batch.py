"""Batched sweeps through the C ABI (lbm_batch_*).

A batch advances many independent cases with the per-node arithmetic of the
single-case step, so every case must match, bit for bit, a context of its own
stepped as often: for every storage format, across CUDA-graph replays and
direct steps, and for every plan (tile width, planes per work item, blocks per
SM) the autotuner may pick.  A subsample is also checked against the FP64
oracle with the float32 parity bounds of the single-case tests.
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


def small_sweep(storage, n=10, seed_offset=7):
    """Cases of every size class (nx <= 96, <= 192, <= 384, > 384), both kinds."""
    r = C.rng(seed_offset)
    sizes = [40, 64, 97, 150, 200, 260, 390, 33, 120, 70][:n]
    out = []
    for i, L in enumerate(sizes):
        kind = i % 2
        p, phi, u, ps = C.sweep_case(kind, L, float(np.exp(r.uniform(np.log(10), np.log(1000)))),
                                     float(np.exp(r.uniform(np.log(1e-5), np.log(1e-3)))),
                                     R=float(r.uniform(8.0, max(8.0, 0.3 * L))))
        p["storage"] = storage
        out.append((p, phi, u, ps))
    return out


def run_single(lib, case, steps):
    p, phi, u, ps = case
    sim = lib.LBM(p)
    sim.init_fields(phi, u, ps)
    sim.step(steps)
    out = sim.fields()
    sim.close()
    return out


def make_batch(lib, cases):
    b = lib.Batch([c[0] for c in cases])
    for i, (p, phi, u, ps) in enumerate(cases):
        b.init_fields(i, phi, u, ps)
    return b


@pytest.mark.parametrize("storage", [0, 1])
def test_batch_equals_single_contexts_bitwise(lib, report, storage):
    cases = small_sweep(storage)
    b = make_batch(lib, cases)
    plan = b.plan()
    assert plan["nclasses"] == 4 and sum(plan["ncases"]) == len(cases)
    steps = 37                       # two graph replays of 16 steps and 5 direct steps
    b.step(steps)
    for i, c in enumerate(cases):
        ref = run_single(lib, c, steps)
        got = b.fields(i)
        for a, r in zip(got, ref):
            assert np.array_equal(a, r), i
    d = b.diag(3)
    assert d["finite"] == 1
    b.close()


def test_batch_plans_do_not_change_results(lib):
    cases = small_sweep(0, n=6)
    ref = [run_single(lib, c, 20) for c in cases]
    b = make_batch(lib, cases)
    plan = b.plan()
    for tx, seg, bps in [(32, 5, 1), (128, 64, 2), (64, 16, 3)]:
        plan2 = dict(plan, tile_x=[tx] * plan["nclasses"], seglen=[seg] * plan["nclasses"],
                     blocks_per_sm=[bps] * plan["nclasses"])
        b.set_plan(plan2)
        got = b.plan()
        assert got["tile_x"] == [tx] * plan["nclasses"] and got["seglen"] == [seg] * plan["nclasses"]
    b.step(20)
    for i in range(len(cases)):
        for a, r in zip(b.fields(i), ref[i]):
            assert np.array_equal(a, r), i
    with pytest.raises(lib.LbmError) as e:
        b.set_plan(dict(plan, tile_x=[48] * plan["nclasses"]))
    assert e.value.code == lib.LBM_ERR_ARG
    b.close()


def test_tune_keeps_the_state_and_picks_a_valid_plan(lib, report):
    cases = small_sweep(1, n=8)
    b = make_batch(lib, cases)
    b.step(3)
    plan = b.tune(trial_steps=3)
    for k in range(plan["nclasses"]):
        assert plan["tile_x"][k] in (32, 64, 128)
        assert plan["seglen"][k] in (4, 16, 64)
        assert plan["blocks_per_sm"][k] >= 1
        assert plan["ms_per_step"][k] > 0
        report("batch_tune_class%d" % k, tile_x=plan["tile_x"][k], seglen=plan["seglen"][k],
               bps=plan["blocks_per_sm"][k], ms=plan["ms_per_step"][k])
    b.step(17)
    for i, c in enumerate(cases):
        ref = run_single(lib, c, 20)
        for a, r in zip(b.fields(i), ref):
            assert np.array_equal(a, r), i
    b.close()


def test_batch_3d_equals_single_contexts(lib):
    cases = []
    for n, R in ((16, 5.0), (24, 7.0), (40, 10.0)):
        p, phi, u, ps = C.drop3d(n=n, R=R, rho_ratio=100.0, mu_ratio=10.0, sigma=1e-3)
        cases.append((p, phi, u, ps))
    b = make_batch(lib, cases)
    b.step(18)
    for i, c in enumerate(cases):
        ref = run_single(lib, c, 18)
        for a, r in zip(b.fields(i), ref):
            assert np.array_equal(a, r), i
    b.close()


def test_batch_subsample_against_oracle(lib, report):
    from oracle import oracle
    oracle.build()
    cases = [C.sweep_case(0, 48, 100.0, 1e-4, R=12.0), C.sweep_case(1, 40, 30.0, 3e-4)]
    b = make_batch(lib, cases)
    b.step(100)
    for i, (p, phi, u, ps) in enumerate(cases):
        o = oracle.Oracle(p)
        o.init_fields(phi, u, ps)
        o.step(100)
        rphi, ru, rp = o.fields()
        gphi, gu, gp = b.fields(i)
        e_phi = np.linalg.norm(gphi - rphi) / np.linalg.norm(rphi)
        # u: relative to the capillary velocity sigma / mu_H (u is a residual
        # current in the drop and a small wave motion in the other case)
        u_sig = p["sigma"] / (p["rho_H"] * p["tau_H"] / 3.0)
        e_u = np.abs(gu - ru).max() / u_sig
        report("batch_oracle_case%d" % i, phi_l2=e_phi, u_cap=e_u)
        assert e_phi <= 1e-5
        assert e_u <= 1e-4
    b.close()
