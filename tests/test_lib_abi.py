"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, exports
every symbol the headers in include/ declare, and fails loudly (no fallback) where
there is no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2505_12205_gb300 import build, lbm
    build.build()
    return lbm


def test_library_exports_every_declared_symbol(lib):
    from paper_2505_12205_gb300 import nn
    names = declared_symbols()
    assert set(names) == set(lib.EXPORTS) | set(nn.NN_EXPORTS)
    so = lib.load()
    for n in names:
        assert hasattr(so, n), n


def test_params_struct_layout(lib):
    # natural alignment of the C struct: 16 int32 then 17 doubles
    assert ctypes.sizeof(lib.LbmParams) == 16 * 4 + 17 * 8
    assert lib.LbmParams.rho_L.offset == 64
    assert lib.LbmParams.mu_ratio.offset == 96
    assert ctypes.sizeof(lib.LbmDiagOut) == 4 * 8 + 2 * 8 + 2 * 4 + 8


@pytest.mark.parametrize("change", ["W", "inlet_without_outlet", "diag_every", "mu_ratio", "tau_L", "layout"])
def test_create_rejects_invalid_parameters_before_touching_a_device(lib, change):
    """Parameter validation of lbm_create (W >= 2, an inlet needs the outlet
    opposite, diag_every >= 0, mu_ratio >= 0, tau_L > 0 unless mu_ratio sets
    it) runs before any CUDA call, so it is checked here without a GPU."""
    import lbm_cases as C
    p = C.jet2d(nx=16, ny=16, half_width=3.0, W=4.0)[0]
    if change == "W":
        p["W"] = 1.5
    elif change == "inlet_without_outlet":
        p["bc"] = [0, 0, 2, 1, 0, 0]
    elif change == "diag_every":
        p["diag_every"] = -1
    elif change == "mu_ratio":
        p["mu_ratio"] = -2.0
    elif change == "layout":
        p["layout"] = 2
    else:
        p["tau_L"] = 0.0
    with pytest.raises(lib.LbmError) as e:
        lib.LBM(p)
    assert e.value.code == lib.LBM_ERR_ARG, lib.lbm_last_error()


def test_no_gpu_means_an_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import lbm_cases as C
    with pytest.raises(lib.LbmError) as e:
        lib.LBM(C.base_params(0, 8, 8, 1))
    assert e.value.code == lib.LBM_ERR_CUDA


def test_ptxas_reports_at_most_token_spills(lib):
    """The D3Q19 step is built for three resident blocks per SM (at most 85
    registers); ptxas may spill a little for that (most with the 16-bit
    conversions), never more than 128 bytes a thread."""
    build_dir = os.path.join(ROOT, "paper_2505_12205_gb300", "_build")
    kernel_units = ["lbm_d3q19", "lbm_d3q19_f16", "lbm_d3q19_bf16", "lbm_d2q9", "lbm_batch_d2q9", "lbm_batch_d3q19"]
    logs = [os.path.join(build_dir, n + ".ptxas.log") for n in kernel_units]
    for log in logs:
        txt = open(log).read()
        assert "sm_103a" in txt
        spills = re.findall(r"(\d+) bytes spill stores", txt)
        assert spills and all(int(s) <= 128 for s in spills)


def test_batch_plan_struct_layout(lib):
    import ctypes
    # int32 nclasses, five int32[8] arrays, padding to 8, double[8]
    assert ctypes.sizeof(lib.LbmBatchPlan) == 4 + 5 * 8 * 4 + 4 + 8 * 8
    assert lib.LbmBatchPlan.ms_per_step.offset == 168


def test_batch_rejects_invalid_cases_before_touching_a_device(lib):
    import lbm_cases as C
    good = C.base_params(0, 16, 16, 1)
    cases = []
    p = dict(good); p["bc"] = [0, 0, 2, 3, 0, 0]; cases.append(p)           # inlet/outlet
    p = dict(good); p["lattice"] = 1; p["nz"] = 4; cases.append(p)          # lattice differs from case 0
    p = dict(good); p["storage"] = 2; cases.append(p)                       # bfloat16
    p = dict(good); p["tau_H"] = -1.0; cases.append(p)                      # invalid physics
    for bad in cases:
        lst = [good, bad] if bad.get("lattice") == 1 else [bad]
        with pytest.raises(lib.LbmError) as e:
            lib.Batch(lst)
        assert e.value.code == lib.LBM_ERR_ARG, bad
        assert lib.lbm_batch_last_error() != ""
    with pytest.raises(lib.LbmError) as e:
        lib.Batch([])
    assert e.value.code == lib.LBM_ERR_ARG
