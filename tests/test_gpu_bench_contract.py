"""bench.py's JSON line on a reduced grid of its workloads: the keys and
objects its consumers read (roofline, e2e, clocks, launches), values that
are finite and consistent with one another."""
import json
import math
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*args):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("args,Q,launches_per_step", [
    (("--grid", "64", "64", "128"), 19, 2),          # k_step_fused + k_faces
    (("--workload", "rt2d", "--grid", "512", "1024", "1"), 9, 1),
])
def test_bench_line(args, Q, launches_per_step):
    steps = 6
    d = run(*args, "--steps", str(steps), "--warmup", "3", "--no-cpu-baseline")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["metric"] == "MLUPS" and d["n_gpus"] == 1 and d["steps"] == steps
    nodes = d["config"]["nodes_per_gpu"]
    assert math.isclose(d["value"], nodes / (d["ms_per_step"] * 1e-3) / 1e6, rel_tol=1e-6)
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["algorithmic_bytes_per_lu"] == 4 * Q * 4
    assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-9)
    assert 0.0 < r["frac"] < 1.5
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0 and e["fields_finite"]
    assert d["gpu_launches"] == launches_per_step * steps
