#!/usr/bin/env python
"""Throughput of the fused phase-field WMRT lattice Boltzmann step on GB300.

Workload: the 3D liquid jet of the paper's application section on D3Q19,
256 x 256 x 1024 nodes (67.1 M), float32 arithmetic and storage, circular plug
inlet (R = 16, u_j = 0.05, We = 2.2, Re = 200, rho* = 100, mu* = 10, W = 5),
convective outlet, periodic sides, gravity along the jet.  One bench step is
one time step of the whole hot path over the grid (the single-pass fused
kernel that recomputes phi, collides and streams, then the inlet and outlet
face kernels).

Output: one JSON line (rank 0).  `value` is whole-job MLUPS (lattice node
updates of both population sets per second) with the state resident in HBM;
`e2e` is the same metric through the C ABI with host buffers (fields copied
in from pinned host memory, fields copied back, both inside the timed
region); `roofline` relates the fused kernel's algorithmic bytes to its
CUDA-event duration and the measured HBM copy bandwidth; `cpu_baseline` times
the FP64 oracle on a slab of the same workload on the host cores.

`--impl reference` times the FP64 CPU oracle (the baseline of this project)
on a bounded slab of the same workload instead.

`--workload rt2d` times the D2Q9 step the same way on the 2D Rayleigh-Taylor
physics (At = 0.5, Re = 3000, W = 5, the 256 x 1024 case) repeated 32 times along
x on an 8192 x 32768 domain (268 M nodes, 38.7 GB of float32 populations).

`--workload learned` measures the learned fast-forward of planar-jet sweeps
(D2Q9 512 x 2048, We in [1, 10]): snapshots generated by the solver, the
network trained on the GPU by the library's kernels, then held-out cases run
with the network in the loop against the solver alone.

`--workload nn` times the learned fast-forward's network alone (inference and
one training step on a 128 x 512 coarse field) against the measured bf16
tensor peak.

`--workload jet-sweep` runs the 3D jet of the application section in the
paper's domain shape (6D x 6D x 20D, D = 32: 192 x 192 x 640, free-slip
sides, plug inlet, convective outlet) for Weber numbers around the critical
one and reports the breakup length and drop size of each (lbm_jet_stats).

`--workload sweep` measures the batched sweep instead: 512 seeded 2D cases
(drops and capillary waves, L x L with L uniform in 64..512, about 51 M nodes,
float16 storage by default) advanced together by the batch API, reported as
cases per hour of 5000 steps, beside the same cases stepped one context per
case (one launch per case and step) on the same GPU.

Multi-GPU (torchrun): independent replicas, one per GPU (weak scaling); the
only collectives are the timing barrier and the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lbm_cases as C  # noqa: E402

WORKLOAD = dict(name="jet3d_D3Q19_256x256x1024_fp32", nx=256, ny=256, nz=1024, Rn=16.0, We=2.2)
SAMPLE_NZ = 8          # slab of the same workload for the CPU oracle
# 2D Rayleigh-Taylor (At = 0.5, Re = 3000, W = 5, the physics of the 256 x 1024
# case) repeated 32 times along x on an 8192 x 32768 domain: 268 M nodes,
# 38.7 GB of float32 populations, the D2Q9 throughput workload
RT_WORKLOAD = dict(name="rt2d_D2Q9_8192x32768", L=256, periods=32, height=32768)
SAMPLE_RT_HEIGHT = 64  # strip of the same workload for the CPU oracle
BYTES_PER_LU = 4 * 19 * 4   # f and g read + written once, float32, D3Q19
METRIC = "MLUPS"
NOMINAL_HBM_GBS = 7900.0    # HBM3e nominal bandwidth of one GB300 (the measured copy peak is the roofline)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("lbm_kernels.cuh", "lbm_lattice.cuh"):
        with open(os.path.join(ROOT, "paper_2505_12205_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload):
    """DRAM bytes per launch of the fused kernel on the full workload from the
    committed ncu summary, if it was taken on the current kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        if d.get("source_sha256_16") == kernel_source_hash():
            return float(d["workloads"][workload]["dram_bytes_per_launch_full_workload"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float) -> float:
    """Max of a per-rank float over the process group (identity without one).
    The only collective of the bench besides the timing barrier; works on the
    nccl (CUDA tensor) and gloo (CPU tensor) backends."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(workload):
    """(params, phi, u, p*, description) of the bounded sample the CPU oracle is timed on."""
    if workload == "rt2d":
        p, phi, u, ps = C.rayleigh_taylor2d(L=RT_WORKLOAD["L"], periods=RT_WORKLOAD["periods"],
                                            height=SAMPLE_RT_HEIGHT)
        return p, phi, u, ps, "strip %dx%d of the Rayleigh-Taylor workload (same parameters, walls)" % (
            p["nx"], p["ny"])
    p, phi, u, ps = C.jet3d(nx=WORKLOAD["nx"], ny=WORKLOAD["ny"], nz=SAMPLE_NZ,
                            Rn=WORKLOAD["Rn"], We=WORKLOAD["We"], stub=4.0)
    return p, phi, u, ps, "slab %dx%dx%d of the jet workload (same parameters, inlet + outlet)" % (
        WORKLOAD["nx"], WORKLOAD["ny"], SAMPLE_NZ)


def oracle_baseline(min_seconds=10.0, max_steps=400, steps=None, workload="jet"):
    """FP64 oracle on a bounded sample of the workload, on all host cores."""
    from oracle import oracle
    p, phi, u, ps, what = oracle_sample(workload)
    o = oracle.Oracle(p)
    o.init_fields(phi, u, ps)
    nodes = p["nx"] * p["ny"] * p["nz"]
    o.step(1)                               # warm-up (page faults)
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(1)
        n += 1
        el = time.perf_counter() - t0
        if steps is not None and n >= steps:
            break
        if steps is None and (el >= min_seconds or n >= max_steps):
            break
    el = time.perf_counter() - t0
    o.close()
    return nodes * n / el / 1e6, n, el, oracle.threads(), nodes, what


def oracle_one_thread(workload, seconds=6.0):
    """The same oracle sample on one host thread (serial), in a fresh process
    with OMP_NUM_THREADS=1: MLUPS, or None if that run fails."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "r = bench.oracle_baseline(min_seconds=%r, max_steps=200, workload=%r); "
            "print(json.dumps({'mlups': r[0], 'steps': r[1], 'seconds': r[2], 'threads': r[3]}))"
            % (ROOT, seconds, workload))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=300).stdout
        d = json.loads(out.strip().splitlines()[-1])
        return {"value": d["mlups"], "unit": "MLUPS", "cores": d["threads"],
                "sample": "the same sample, %d steps, %.1f s" % (d["steps"], d["seconds"])}
    except Exception:
        return None


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    try:
        from oracle import oracle
        oracle.build()
    except Exception as e:  # pragma: no cover
        print(json.dumps({"impl": "reference", "unavailable": "oracle build failed: %s" % e}))
        return 0
    for _ in range(max(args.warmup, 0)):
        pass
    mlups, n, el, cores, nodes, what = oracle_baseline(steps=max(args.steps, 1), workload=args.workload)
    sample = "%s, %d steps" % (what, n)
    name = RT_WORKLOAD["name"] + "_" + (args.storage or "fp32") if args.workload == "rt2d" else WORKLOAD["name"]
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / n * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "sample_nodes": nodes},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2505_12205_gb300 import build, lbm
    build.build()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import oracle
        oracle.build()
        mlups, n, el, cores, nodes, what = oracle_baseline(workload=args.workload)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": "%s, %d steps, %.1f s" % (what, n, el),
               "one_thread": oracle_one_thread(args.workload)}

    rt = args.workload == "rt2d"
    if rt:
        L = RT_WORKLOAD["L"]
        per, height = (args.grid[0] // L, args.grid[1]) if args.grid else (RT_WORKLOAD["periods"],
                                                                          RT_WORKLOAD["height"])
        p, phi, u, ps = C.rayleigh_taylor2d(L=L, periods=per, height=height)
        Q, dim, lat, faces = 9, 2, "D2Q9", 0
        name = "rt2d_D2Q9_%dx%d_%s" % (p["nx"], p["ny"], args.storage)
        kname = "k_step_fused<D2Q9,64,1> (phi + collide + push-stream, one pass)"
        extra = {"At": 0.5, "Re": 3000.0, "W": 5.0,
                 "note": "Rayleigh-Taylor physics of the 256 x 1024 case repeated %d times along x" % per}
    else:
        nx, ny, nz = args.grid if args.grid else (WORKLOAD["nx"], WORKLOAD["ny"], WORKLOAD["nz"])
        p, phi, u, ps = C.jet3d(nx=nx, ny=ny, nz=nz, Rn=WORKLOAD["Rn"], We=WORKLOAD["We"])
        Q, dim, lat, faces = 19, 3, "D3Q19", 1          # k_faces: inlet + outlet in one launch
        name = WORKLOAD["name"] if not args.grid else "jet3d_D3Q19_%dx%dx%d_fp32 (reduced grid)" % tuple(args.grid)
        if args.storage != "fp32":
            name = name.replace("fp32", args.storage)
        kname = "k_step_fused<D3Q19,32,6> (phi + collide + push-stream, one pass)"
        extra = {"We": WORKLOAD["We"]}
    p["storage"] = {"fp32": 0, "fp16": 1, "bf16": 2}[args.storage]
    if args.storage != "fp32":
        # 16-bit storage: the A/B step holds two x-adjacent nodes per thread
        kname = (("k_step_fused2<D2Q9,64,1> (phi + collide + push-stream, one pass, two nodes per thread)") if rt else
                 ("k_step_fused2<D3Q19,64,4> (phi + collide + push-stream, one pass, two nodes per thread)"))
    inplace = args.layout == "inplace"
    p["layout"] = 1 if inplace else 0
    p["diag_every"] = args.diag_every
    if inplace:
        name += " (in-place layout)"
        kname = ("k_step_inplace<D2Q9,64,1>" if rt else "k_step_inplace<D3Q19,32,6>") + \
            " (collide + in-place stream, even/odd forms; phi by a pre-pass)"
    elem = 4 if args.storage == "fp32" else 2
    N = p["nx"] * p["ny"] * p["nz"]
    stream = torch.cuda.current_stream()
    sim = lbm.LBM(p, stream=stream)
    phi_d = torch.from_numpy(phi).cuda()
    u_d = torch.from_numpy(u).cuda()
    sim.init_fields(phi_d, u_d, None)
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()

    # ---------------- device-resident timed region
    sim.set_timing(True)
    sim.timing()
    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sim.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_phi, ms_step, ms_face, nrec = sim.timing()
    sim.set_timing(False)
    ms_max = max_over_ranks(ms)
    value = N * args.steps * ws / (ms_max * 1e-3) / 1e6

    # roofline of the fused collide-stream kernel
    peak, peak_kind = peaks()
    step_ms = ms_step / max(nrec, 1)
    bytes_per_lu = 4 * Q * elem
    achieved = bytes_per_lu * N / (step_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "frac_of_nominal_7900": achieved / NOMINAL_HBM_GBS,
            "traffic": (ncu_traffic(args.workload + ("" if args.storage == "fp32" else "_" + args.storage))
                        if (args.storage in ("fp32", "fp16") and not args.grid and not inplace) else None),
            "kernel": kname,
            "phi_prepass_ms_per_step": ms_phi / max(nrec, 1),
            "algorithmic_bytes_per_lu": bytes_per_lu, "peak_source": peak_kind + " hbm_gbs",
            "kernel_share_of_step": ms_step / max(ms_phi + ms_step + ms_face, 1e-9)}

    # ---------------- end to end through the C ABI with host buffers
    phi_h = torch.from_numpy(phi).pin_memory()
    u_h = torch.from_numpy(u).pin_memory()
    ps_h = torch.zeros(N, dtype=torch.float32).pin_memory()
    o_phi = torch.empty(N, dtype=torch.float32).pin_memory()
    o_u = torch.empty(dim * N, dtype=torch.float32).pin_memory()
    o_p = torch.empty(N, dtype=torch.float32).pin_memory()
    # warm-up of lbm_step's graph replay (its first use captures the graphs;
    # the timed run below starts from freshly initialised fields)
    lbm.lbm_step(sim._h, 32)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    lbm.lbm_init_fields(sim._h, phi_h, u_h, ps_h, n=N, dim=dim)
    lbm.lbm_step(sim._h, args.steps)
    lbm.lbm_get_fields(sim._h, o_phi, o_u, o_p)
    te2e = time.perf_counter() - t0
    te2e = max_over_ranks(te2e)
    ok = bool(np.isfinite(o_phi.numpy()).all())
    h2d = (phi_h.numel() + u_h.numel() + ps_h.numel()) * 4
    d2h = (o_phi.numel() + o_u.numel() + o_p.numel()) * 4
    e2e = {"value": N * args.steps * ws / te2e / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "fields_finite": ok,
           "note": "one job per rank: fields in from pinned host, %d steps, fields back" % args.steps}
    sim.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage == "fp32" else "f32 arithmetic, %s storage" % args.storage,
            "data": "synthetic",
            "config": dict({"workload": name, "lattice": lat,
                            "grid": [p["nx"], p["ny"], p["nz"]], "nodes_per_gpu": N,
                            "storage": args.storage,
                            "layout": "in place (one copy)" if inplace else "A/B (two copies)",
                            "diag_every": args.diag_every,
                            "l2": "inputs larger than L2: %.1f GB of populations per GPU vs 129 MB L2"
                                  % ((2 if inplace else 4) * Q * elem * N / 1e9),
                            "parallelism": "replicas" if ws > 1 else "single"}, **extra),
            "hbm_gbs_algorithmic": value / ws * 1e6 * bytes_per_lu / 1e9 if ws == 1 else None,
            "roofline": roof,
            "e2e": e2e,
            # per step: the fused kernel (+ the phi pre-pass in place) and the
            # face kernels; per in-step diagnostic: k_phi, k_diag, k_diag_final
            "gpu_launches": (1 + (1 if inplace else 0) + faces) * args.steps
                            + (3 * (args.steps // args.diag_every) if args.diag_every else 0),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


SWEEP = dict(name="sweep512_D2Q9_L64-512_drop+capillary-wave", ncases=512, steps_per_case=5000)


def run_sweep(args):
    """Cases per hour of the batched sweep vs one context per case."""
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2505_12205_gb300 import build, lbm
    build.build()
    storage = {"fp32": 0, "fp16": 1, "bf16": 2}[args.storage or "fp16"]
    if storage == 2:
        raise SystemExit("the batched sweep stores float32 or float16")
    elem = 4 if storage == 0 else 2
    cases = C.sweep_cases(n=SWEEP["ncases"], seed_offset=4 + rank)
    for c in cases:
        c[0]["storage"] = storage
    nodes = sum(c[0]["nx"] * c[0]["ny"] for c in cases)
    ncases = len(cases)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import oracle
        oracle.build()
        p, phi, u, ps = C.sweep_case(0, 256, 100.0, 1e-4, R=60.0)
        o = oracle.Oracle(p)
        o.init_fields(phi, u, ps)
        o.step(1)
        t0, n = time.perf_counter(), 0
        while time.perf_counter() - t0 < 10.0 and n < 2000:
            o.step(1)
            n += 1
        el = time.perf_counter() - t0
        o.close()
        mlups_cpu = 256 * 256 * n / el / 1e6
        cph_cpu = ncases * 3600.0 / (nodes * SWEEP["steps_per_case"] / (mlups_cpu * 1e6))
        cpu = {"value": cph_cpu, "unit": "cases/h", "cores": oracle.threads(), "kind": "oracle",
               "sample": "one 256x256 drop case of the sweep, %d steps, %.1f s (%.2f MLUPS), scaled to the "
                         "sweep's %d nodes x %d steps" % (n, el, mlups_cpu, nodes, SWEEP["steps_per_case"])}

    stream = torch.cuda.current_stream()
    batch = lbm.Batch([c[0] for c in cases], stream=stream)
    for i, (p, phi, u, ps) in enumerate(cases):
        batch.init_fields(i, phi, u, ps)
    plan = batch.tune(trial_steps=3)
    batch.step(max(args.warmup, 3))
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    ms_step = ms / args.steps
    cph = ws * ncases * 3600.0 / (ms_step * 1e-3 * SWEEP["steps_per_case"])
    finite = all(batch.diag(i)["finite"] == 1 for i in range(0, ncases, 37))

    # the same cases, one context each, stepped in turn (one launch per case and step)
    sims = []
    for p, phi, u, ps in cases:
        s = lbm.LBM(p, stream=stream)
        s.init_fields(phi, u, ps)
        sims.append(s)
    for s in sims:
        s.step(1)
    torch.cuda.synchronize()
    kp = max(2, args.steps // 10)
    e0.record(stream)
    for _ in range(kp):
        for s in sims:
            s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = max_over_ranks(e0.elapsed_time(e1)) / kp
    for s in sims:
        s.close()
    cph_plain = ws * ncases * 3600.0 / (ms_plain * 1e-3 * SWEEP["steps_per_case"])

    # end to end through the C ABI with host buffers: fields of every case in,
    # the steps, fields of every case out
    hostf = [(torch.from_numpy(phi).pin_memory(), torch.from_numpy(u).pin_memory()) for _, phi, u, _ in cases]
    outs = [(torch.empty(c[0]["nx"] * c[0]["ny"], dtype=torch.float32).pin_memory(),
             torch.empty(2 * c[0]["nx"] * c[0]["ny"], dtype=torch.float32).pin_memory()) for c in cases]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, (ph, uu) in enumerate(hostf):
        lbm.lbm_batch_init_fields(batch._h, i, ph, uu, None)
    batch.step(args.steps)
    for i, (oph, ou) in enumerate(outs):
        lbm.lbm_batch_get_fields(batch._h, i, oph, ou, None)
    te2e = max_over_ranks(time.perf_counter() - t0)
    h2d = sum((a.numel() + b.numel()) * 4 for a, b in hostf)
    d2h = sum((a.numel() + b.numel()) * 4 for a, b in outs)
    batch.close()

    bytes_per_lu = 4 * 9 * elem
    peak, peak_kind = peaks()
    achieved = bytes_per_lu * nodes / (ms_step * 1e-3) / 1e9
    if rank == 0:
        line = {
            "metric": "cases_per_hour", "value": cph, "unit": "cases/h", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 arithmetic, %s storage" % ("fp16" if storage else "fp32"),
            "data": "synthetic",
            "config": {"workload": SWEEP["name"], "cases": ncases, "nodes": nodes,
                       "steps_per_case": SWEEP["steps_per_case"], "storage": "fp16" if storage else "fp32",
                       "l2": "inputs larger than L2: %.2f GB of populations vs 129 MB L2"
                             % (4 * 9 * elem * nodes / 1e9),
                       "plan": plan, "parallelism": "replicas" if ws > 1 else "single"},
            "mlups": nodes * ws / (ms_step * 1e-3) / 1e6,
            "plain": {"value": cph_plain, "unit": "cases/h", "ms_per_step_all_cases": ms_plain,
                      "note": "one context per case, every case stepped in turn (one launch per case and step)"},
            "speedup_vs_plain": cph / cph_plain,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "frac_of_nominal_7900": achieved / NOMINAL_HBM_GBS,
                         "traffic": None,
                         "kernel": "k_step_batch<D2Q9> (all classes of one step, concurrent)",
                         "algorithmic_bytes_per_lu": bytes_per_lu, "peak_source": peak_kind + " hbm_gbs"},
            "e2e": {"value": ws * ncases * 3600.0 / (te2e / args.steps * SWEEP["steps_per_case"]),
                    "unit": "cases/h", "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "note": "fields of every case in from pinned host, %d steps, fields back" % args.steps},
            "fields_finite": finite,
            "gpu_launches": plan["nclasses"] * args.steps,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


LEARNED = dict(name="planar-jet fast-forward, D2Q9 512x2048, We in [1,10], K=200",
               train_We=[1.0, 2.3, 3.6, 4.9, 6.1, 7.4, 8.7, 10.0], t0=4000, t1=12000)


def run_learned(args):
    """Cases per hour of planar-jet runs with the learned fast-forward in the
    loop vs the solver alone, on held-out Weber numbers."""
    import torch
    from paper_2505_12205_gb300 import build, nn, surrogate as S
    build.build()
    torch.cuda.set_device(0)
    nn.set_conv_path({"tcgen05": 0, "mma.sync": 1, "auto": 2}[args.conv_path])
    t0, t1 = LEARNED["t0"], LEARNED["t1"]
    log = lambda msg: print("[learned] " + msg, file=sys.stderr, flush=True)
    tic = time.perf_counter()
    X, Y, cases = S.generate(LEARNED["train_We"], t0, t1)
    t_gen = time.perf_counter() - tic
    r = np.random.Generator(np.random.PCG64(C.SEED + 5))
    test_We = sorted(float(w) for w in r.uniform(1.0, 10.0, 4))
    Xt, Yt, _ = S.generate(test_We, t0, t1)
    net = nn.UNet(cin=S.CIN, ch=(32, 64, 128, 256))
    net.init_he(seed=7)
    tic = time.perf_counter()
    hist = S.train(net, X, Y, np.arange(X.shape[0]), epochs=args.epochs, accum=4, lr=1e-3, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - tic
    val, pers = S.evaluate(net, Xt, Yt, np.arange(Xt.shape[0]))
    solves = args.solve or [1]
    res = [S.fast_forward(net, w, t0, t1, skip=args.skip, twins=True, solve=solves[0]) for w in test_We]
    more = []
    for sv in solves[1:]:
        rs = [S.fast_forward(net, w, t0, t1, skip=args.skip, twins=False, solve=sv) for w in test_We]
        more.append({"solve": sv, "skip": args.skip,
                     "speedup_vs_solver": sum(x["ms_solver"] for x in rs) / sum(x["ms_fast_forward"] for x in rs),
                     "accepted_at_end": sum(1 for x in rs if x["accepted_at_end"]),
                     "final_interface_distance": [x["final_interface_distance"] for x in rs],
                     "final_front_error": [x["final_front_error"] for x in rs],
                     "final_mass_error": [x["final_mass_error"] for x in rs],
                     "windows": [x["windows"] for x in rs]})
    ms_solver = sum(x["ms_solver"] for x in res)
    ms_ff = sum(x["ms_fast_forward"] for x in res)
    steps = t1 - t0
    accepted = [x for x in res if x["accepted_at_end"]]
    line = {
        "metric": "cases_per_hour_learned", "value": len(res) * 3600e3 / ms_ff, "unit": "cases/h",
        "n_gpus": 1, "steps": steps, "warmup": 0, "ms_per_step": ms_ff / len(res) / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 solver, bf16 network with f32 accumulation", "data": "synthetic (generated by the solver)",
        "config": {"workload": LEARNED["name"], "train_We": LEARNED["train_We"], "test_We": test_We,
                   "span_steps": [t0, t1], "pairs": int(X.shape[0]), "epochs": args.epochs, "skip": args.skip,
                   "solve": solves[0],
                   "network": "4-level encoder-decoder, channels 32-256, 128x512 input"},
        "solver_alone": {"value": len(res) * 3600e3 / ms_solver, "unit": "cases/h"},
        "speedup_vs_solver": ms_solver / ms_ff,
        "accepted_at_end": len(accepted), "cases": len(res),
        "final_interface_distance": {
            "network_in_the_loop": [x["final_interface_distance"] for x in res],
            "solver_perturbed_1e-6": [x["twin_perturb"]["final_interface_distance"] for x in res],
            "solver_restarted_from_itself": [x["twin_restart"]["final_interface_distance"] for x in res]},
        "train": {"seconds": t_train, "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                  "generate_seconds": t_gen},
        "held_out": {"loss": val, "persistence_loss": pers},
        "per_case": [{k: v for k, v in x.items() if k != "judged"} for x in res],
        "other_solve_counts": more,
        "judged_windows": [[{k: (round(v, 4) if v is not None else None) for k, v in j.items()} for j in x["judged"]]
                           for x in res],
    }
    print(json.dumps(line))
    return 0


def unet_flops(cin, ch, head, H, W):
    """Multiply-adds x 2 of one forward pass of the encoder-decoder (3x3
    convolutions with zero padding, 1x1 head) on an H x W input."""
    macs, L = 0, len(ch)
    for l in range(L):
        c_in = cin if l == 0 else ch[l - 1]
        macs += (H >> l) * (W >> l) * 9 * (c_in * ch[l] + ch[l] * ch[l])
    for l in range(L - 2, -1, -1):
        macs += (H >> l) * (W >> l) * 9 * ((ch[l + 1] + ch[l]) * ch[l] + ch[l] * ch[l])
    macs += H * W * ch[0] * head
    return 2 * macs


def run_nn(args):
    """Throughput of the learned fast-forward's network (the encoder-decoder
    of the learned workload on one 128 x 512 coarse field): inference and one
    training step (forward, backward-data and weight gradients), bfloat16
    tensor-core convolutions with float32 accumulation."""
    import torch
    from paper_2505_12205_gb300 import build, nn
    build.build()
    torch.cuda.set_device(0)
    nn.load()
    cin, ch, head, H, W = 8, (32, 64, 128, 256), 8, 512, 128
    nb = args.batch
    nn.set_conv_path({"tcgen05": 0, "mma.sync": 1, "auto": 2}[args.conv_path])
    net = nn.UNet(cin=cin, ch=ch, head=head)
    net.init_he(seed=7)
    g = torch.Generator(device="cuda")
    g.manual_seed(C.SEED + 9)
    x = (0.5 * torch.randn(nb * H * W, cin, generator=g, device="cuda")).to(torch.bfloat16).contiguous()
    t = torch.randn(nb * H * W, 3, generator=g, device="cuda").contiguous()
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        net.forward(x, nb, H, W, target=t)
        net.backward(x, nb, H, W)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    for _ in range(args.steps):
        net.forward(x, nb, H, W)
    e1.record(stream)
    for _ in range(args.steps):
        net.forward(x, nb, H, W, target=t)
        net.backward(x, nb, H, W)
    e2.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_inf = e0.elapsed_time(e1) / args.steps
    ms_train = e1.elapsed_time(e2) / args.steps
    f_inf = nb * unet_flops(cin, ch, head, H, W)
    timed_out = nn.conv_timed_out()
    tf_inf = f_inf / (ms_inf * 1e-3) / 1e12
    tf_train = 3 * f_inf / (ms_train * 1e-3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, kind = float(json.load(f)["bf16_tflops"]), "measured bf16_tflops (burst)"
    except Exception:
        peak, kind = 1900.0, "fallback"
    line = {"metric": "TFLOP/s", "value": tf_inf, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_inf, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 operands, f32 accumulation", "data": "synthetic",
            "config": {"workload": "encoder-decoder 32-256 channels on %d x 128 x 512 x 8 inputs (learned fast-forward)" % nb,
                       "batch": nb, "conv_path": args.conv_path,
                       "gflop_per_inference": f_inf / 1e9, "l2": "weights and activations are L2-resident"
                       if nb <= 4 else "activations partly beyond L2"},
            "training_step": {"ms": ms_train, "tflops": tf_train},
            "roofline": {"bound": "tensor", "achieved": tf_inf, "peak": peak, "unit": "TFLOP/s",
                         "frac": tf_inf / peak, "traffic": None, "peak_source": kind,
                         "kernel": {"tcgen05": "k_conv_fwd_tc (tcgen05.mma, tensor-memory accumulator)",
                                    "mma.sync": "k_conv_fwd (mma.sync m16n8k16 bf16)",
                                    "auto": "k_conv_fwd_tc (tcgen05) for calls of >= 4 GFLOP, else "
                                            "k_conv_fwd (mma.sync)"}[args.conv_path] + " + split-K reduction"},
            "bounded_wait_timed_out": timed_out,
            "clocks": clk}
    print(json.dumps(line))
    return 0


JETSWEEP = dict(We=[1.0, 2.2, 3.5, 5.0, 10.0], nx=192, ny=192, nz=640, Rn=16.0, steps=48000, sample_from=24000,
                sample_every=500)


def run_jet_sweep(args):
    """Breakup length L_b / D and mean drop diameter d_e / D against We."""
    import torch
    from paper_2505_12205_gb300 import build, lbm
    build.build()
    torch.cuda.set_device(0)
    cfg = JETSWEEP
    D = 2.0 * cfg["Rn"]
    rows = []
    tic = time.perf_counter()
    for We in (args.we if args.we else cfg["We"]):
        p, phi, u, ps = C.jet3d(nx=cfg["nx"], ny=cfg["ny"], nz=cfg["nz"], Rn=cfg["Rn"], We=We)
        p["bc"] = [C.FREESLIP, C.FREESLIP, C.FREESLIP, C.FREESLIP, C.INLET, C.OUTFLOW]
        sim = lbm.LBM(p)
        sim.init_fields(phi, u, ps)
        sim.step(cfg["sample_from"])
        Lb, de, nd = [], [], []
        t = cfg["sample_from"]
        while t < cfg["steps"]:
            sim.step(cfg["sample_every"])
            t += cfg["sample_every"]
            st = sim.jet_stats(0.5)
            Lb.append(st["breakup_length"] / D)
            nd.append(st["n_drops"])
            if st["n_drops"]:
                de.append(st["mean_drop_diameter"] / D)
        finite = sim.diag()["finite"] == 1
        sim.close()
        rows.append(dict(We=We, breakup_length_over_D=float(np.mean(Lb)), breakup_length_std=float(np.std(Lb)),
                         drop_diameter_over_D=float(np.mean(de)) if de else None, drops_mean=float(np.mean(nd)),
                         samples=len(Lb), finite=bool(finite)))
    line = {"metric": "jet_breakup_vs_We", "value": None, "unit": "L_b/D", "n_gpus": 1,
            "steps": cfg["steps"], "higher_is_better": None, "data": "synthetic",
            "config": {"workload": "3D jet 6Dx6Dx20D (D = 32), free-slip sides, Re = 200, rho* = 100, mu* = 10",
                       "grid": [cfg["nx"], cfg["ny"], cfg["nz"]], "sampled_steps": [cfg["sample_from"], cfg["steps"]],
                       "sample_every": cfg["sample_every"]},
            "seconds": time.perf_counter() - tic, "rows": rows}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--storage", default=None, choices=["fp32", "fp16", "bf16"],
                    help="population storage format (arithmetic is float32); default fp32 for the "
                         "jet, fp16 for the sweep")
    ap.add_argument("--workload", default="jet", choices=["jet", "rt2d", "sweep", "learned", "jet-sweep", "nn"])
    ap.add_argument("--batch", type=int, default=1, help="inputs per inference of the nn workload")
    ap.add_argument("--conv-path", default="auto", choices=["auto", "tcgen05", "mma.sync"],
                    help="convolution contraction of the nn / learned workloads (auto: tcgen05 for large calls)")
    ap.add_argument("--we", type=float, nargs="+", default=None,
                    help="Weber numbers of the jet-sweep workload (default: 1, 2.2, 3.5, 5, 10)")
    ap.add_argument("--layout", default="ab", choices=["ab", "inplace"],
                    help="population layout of the jet / rt2d workloads: two copies (A/B) or one (in place)")
    ap.add_argument("--diag-every", type=int, default=100,
                    help="steps between the in-step FP64 diagnostics (sum phi, finite check) of lbm_step")
    ap.add_argument("--epochs", type=int, default=24, help="training epochs of the learned workload")
    ap.add_argument("--skip", type=int, default=1, help="windows predicted after each passing check (learned)")
    ap.add_argument("--solve", type=int, nargs="+", default=None,
                    help="solver windows required since the last skip before the next (learned; several values: "
                         "one training, a fast-forward run per value)")
    ap.add_argument("--grid", type=int, nargs=3, metavar=("NX", "NY", "NZ"), default=None,
                    help="reduced grid of the same jet workload (profiling captures); for rt2d NX "
                         "(a multiple of 256) and NY, NZ ignored")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "nn":
        return run_nn(args)
    if args.workload == "jet-sweep":
        return run_jet_sweep(args)
    if args.storage is None:
        args.storage = "fp32"
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
