"""Thin ctypes binding of the C ABI in ``include/lbm.h``.

The module-level functions carry the C names (``lbm_create``,
``lbm_init_fields``, ``lbm_step``, ``lbm_get_fields``, ``lbm_destroy``, ...)
and only marshal arguments: host arrays are numpy float32, device arrays are
contiguous float32 CUDA ``torch.Tensor``s (their ``data_ptr()`` is passed with
``on_device = 1``).  Every step of the method runs in the CUDA library; there
is no Python or CPU fallback, and loading fails loudly when the library has
not been built.  ``LBM`` wraps one context for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm.so")

LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_BC_PERIODIC, LBM_BC_WALL, LBM_BC_INLET, LBM_BC_OUTFLOW, LBM_BC_FREESLIP = 0, 1, 2, 3, 4
LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT, LBM_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6

# every symbol declared in include/lbm.h
EXPORTS = ["lbm_create", "lbm_init_fields", "lbm_step", "lbm_get_fields", "lbm_get_populations",
           "lbm_set_populations", "lbm_diag", "lbm_sync", "lbm_shape", "lbm_last_error",
           "lbm_destroy", "lbm_collide_cells", "lbm_set_timing", "lbm_get_timing",
           "lbm_diag_noalloc", "lbm_diag_last", "lbm_advect_phase", "lbm_jet_stats", "lbm_batch_create", "lbm_batch_init_fields", "lbm_batch_step",
           "lbm_batch_get_fields", "lbm_batch_diag", "lbm_batch_get_plan", "lbm_batch_set_plan",
           "lbm_batch_tune", "lbm_batch_sync", "lbm_batch_last_error", "lbm_batch_destroy"]

LBM_BATCH_MAX_CLASSES = 8


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 6),
        ("visc_model", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("outlet_scheme", ctypes.c_int32), ("diag_every", ctypes.c_int32),
        ("layout", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("rho_L", ctypes.c_double), ("rho_H", ctypes.c_double),
        ("tau_L", ctypes.c_double), ("tau_H", ctypes.c_double),
        ("mu_ratio", ctypes.c_double),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double),
        ("mobility", ctypes.c_double),
        ("force", ctypes.c_double * 3), ("rho_ref", ctypes.c_double),
        ("inlet_u", ctypes.c_double),
        ("inlet_center", ctypes.c_double * 2),
        ("inlet_radius", ctypes.c_double),
        ("storage_scale", ctypes.c_double),
    ]


class LbmDiagOut(ctypes.Structure):
    _fields_ = [
        ("sum_phi", ctypes.c_double), ("sum_p_in", ctypes.c_double),
        ("sum_p_out", ctypes.c_double), ("max_speed", ctypes.c_double),
        ("n_in", ctypes.c_int64), ("n_out", ctypes.c_int64),
        ("finite", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("dp_laplace", ctypes.c_double),
    ]


class LbmJetStats(ctypes.Structure):
    _fields_ = [
        ("n_components", ctypes.c_int32), ("has_jet", ctypes.c_int32),
        ("breakup_length", ctypes.c_double),
        ("n_drops", ctypes.c_int32), ("truncated", ctypes.c_int32),
        ("mean_drop_diameter", ctypes.c_double), ("drop_volume", ctypes.c_double),
    ]


class LbmBatchPlan(ctypes.Structure):
    _fields_ = [
        ("nclasses", ctypes.c_int32),
        ("nx_max", ctypes.c_int32 * LBM_BATCH_MAX_CLASSES),
        ("ncases", ctypes.c_int32 * LBM_BATCH_MAX_CLASSES),
        ("tile_x", ctypes.c_int32 * LBM_BATCH_MAX_CLASSES),
        ("seglen", ctypes.c_int32 * LBM_BATCH_MAX_CLASSES),
        ("blocks_per_sm", ctypes.c_int32 * LBM_BATCH_MAX_CLASSES),
        ("ms_per_step", ctypes.c_double * LBM_BATCH_MAX_CLASSES),
    ]


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lbm error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (built in-tree by ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: run paper_2505_12205_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    vp, f32p, i64, i32p = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
    P = ctypes.POINTER(LbmParams)
    lib.lbm_create.argtypes = [P, vp, ctypes.POINTER(vp)]
    lib.lbm_init_fields.argtypes = [vp, f32p, f32p, f32p, ctypes.c_int]
    lib.lbm_step.argtypes = [vp, i64]
    lib.lbm_get_fields.argtypes = [vp, f32p, f32p, f32p, ctypes.c_int]
    lib.lbm_get_populations.argtypes = [vp, f32p, f32p, ctypes.c_int]
    lib.lbm_set_populations.argtypes = [vp, f32p, f32p, ctypes.c_int]
    lib.lbm_diag.argtypes = [vp, ctypes.c_double, ctypes.POINTER(LbmDiagOut)]
    lib.lbm_sync.argtypes = [vp]
    lib.lbm_shape.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), i32p]
    lib.lbm_last_error.argtypes = [vp]
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_destroy.argtypes = [vp]
    lib.lbm_collide_cells.argtypes = [P, i64, f32p, f32p, f32p, f32p, f32p, f32p, vp]
    lib.lbm_diag_noalloc.argtypes = [P, f32p, f32p, ctypes.c_double, ctypes.POINTER(LbmDiagOut), vp]
    lib.lbm_diag_last.argtypes = [vp, ctypes.POINTER(LbmDiagOut), ctypes.POINTER(ctypes.c_int64)]
    lib.lbm_set_timing.argtypes = [vp, ctypes.c_int]
    lib.lbm_advect_phase.argtypes = [vp, f32p, ctypes.c_double, i64, ctypes.c_int]
    lib.lbm_jet_stats.argtypes = [vp, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(LbmJetStats)]
    lib.lbm_get_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    BP = ctypes.POINTER(LbmBatchPlan)
    lib.lbm_batch_create.argtypes = [P, ctypes.c_int32, vp, ctypes.POINTER(vp)]
    lib.lbm_batch_init_fields.argtypes = [vp, ctypes.c_int32, f32p, f32p, f32p, ctypes.c_int32]
    lib.lbm_batch_step.argtypes = [vp, i64]
    lib.lbm_batch_get_fields.argtypes = [vp, ctypes.c_int32, f32p, f32p, f32p, ctypes.c_int32]
    lib.lbm_batch_diag.argtypes = [vp, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(LbmDiagOut)]
    lib.lbm_batch_get_plan.argtypes = [vp, BP]
    lib.lbm_batch_set_plan.argtypes = [vp, BP]
    lib.lbm_batch_tune.argtypes = [vp, ctypes.c_int32, BP]
    lib.lbm_batch_sync.argtypes = [vp]
    lib.lbm_batch_last_error.argtypes = [vp]
    lib.lbm_batch_destroy.argtypes = [vp]
    for name in EXPORTS:
        text = name in ("lbm_last_error", "lbm_batch_last_error")
        getattr(lib, name).restype = ctypes.c_char_p if text else ctypes.c_int
    _lib = lib
    return lib


def make_params(p: dict) -> LbmParams:
    s = LbmParams()
    s.lattice = int(p["lattice"])
    s.nx, s.ny, s.nz = int(p["nx"]), int(p["ny"]), int(p.get("nz", 1))
    for i, b in enumerate(p.get("bc", [0] * 6)):
        s.bc[i] = int(b)
    s.visc_model = int(p.get("visc_model", 0))
    s.storage = int(p.get("storage", 0))
    s.outlet_scheme = int(p.get("outlet_scheme", 0))
    s.diag_every = int(p.get("diag_every", 0))
    s.layout = int(p.get("layout", 0))
    s.rho_L, s.rho_H = float(p["rho_L"]), float(p["rho_H"])
    s.tau_L, s.tau_H = float(p.get("tau_L", 0.0)), float(p["tau_H"])
    s.mu_ratio = float(p.get("mu_ratio", 0.0))
    s.sigma, s.W, s.mobility = float(p["sigma"]), float(p["W"]), float(p["mobility"])
    g = list(p.get("force", (0.0, 0.0, 0.0))) + [0.0] * 3
    for i in range(3):
        s.force[i] = float(g[i])
    s.rho_ref = float(p.get("rho_ref", 0.0))
    s.inlet_u = float(p.get("inlet_u", 0.0))
    c = list(p.get("inlet_center", (0.0, 0.0))) + [0.0, 0.0]
    s.inlet_center[0], s.inlet_center[1] = float(c[0]), float(c[1])
    s.inlet_radius = float(p.get("inlet_radius", 0.0))
    s.storage_scale = float(p.get("storage_scale", 0.0))
    return s


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, n_expected=None):
    """(address, on_device) of a float32 array: numpy (host) or torch CUDA tensor."""
    if a is None:
        return None, None
    if _is_torch(a):
        if a.dtype.__str__() != "torch.float32" or not a.is_contiguous():
            raise ValueError("device arrays must be contiguous float32 tensors")
        if n_expected is not None and a.numel() != n_expected:
            raise ValueError("array has %d elements, expected %d" % (a.numel(), n_expected))
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous):
        raise ValueError("host arrays must be C-contiguous float32 numpy arrays")
    if n_expected is not None and a.size != n_expected:
        raise ValueError("array has %d elements, expected %d" % (a.size, n_expected))
    return ctypes.c_void_p(a.ctypes.data), 0


def _check(lib, code, ctx=None):
    if code != LBM_OK:
        msg = lib.lbm_last_error(ctx)
        raise LbmError(code, msg.decode() if msg else "")


def _one_kind(*kinds):
    ks = {k for k in kinds if k is not None}
    if len(ks) > 1:
        raise ValueError("mixing host and device arrays in one call")
    return ks.pop() if ks else 0


# ----------------------------------------------------- C-named entry points

def lbm_create(params: dict, stream=None):
    lib = load()
    s = make_params(params)
    h = ctypes.c_void_p()
    st = ctypes.c_void_p(_stream_handle(stream))
    _check(lib, lib.lbm_create(ctypes.byref(s), st, ctypes.byref(h)))
    return h


def lbm_init_fields(ctx, phi, u=None, pstar=None, n=None, dim=None):
    lib = load()
    a, k1 = _ptr(phi, n)
    b, k2 = _ptr(u, None if n is None else n * dim)
    c, k3 = _ptr(pstar, n)
    _check(lib, lib.lbm_init_fields(ctx, a, b, c, _one_kind(k1, k2, k3)), ctx)


def lbm_step(ctx, nsteps: int):
    lib = load()
    _check(lib, lib.lbm_step(ctx, int(nsteps)), ctx)


def _dims(ctx):
    """(N, Q, D) of a context."""
    n, q = lbm_shape(ctx)
    return n, q, 2 if q == 9 else 3


def lbm_get_fields(ctx, phi=None, u=None, p=None):
    lib = load()
    n, _, d = _dims(ctx)
    a, k1 = _ptr(phi, n)
    b, k2 = _ptr(u, n * d)
    c, k3 = _ptr(p, n)
    _check(lib, lib.lbm_get_fields(ctx, a, b, c, _one_kind(k1, k2, k3)), ctx)


def lbm_get_populations(ctx, f=None, g=None):
    lib = load()
    n, q, _ = _dims(ctx)
    a, k1 = _ptr(f, n * q)
    b, k2 = _ptr(g, n * q)
    _check(lib, lib.lbm_get_populations(ctx, a, b, _one_kind(k1, k2)), ctx)


def lbm_set_populations(ctx, f, g):
    lib = load()
    n, q, _ = _dims(ctx)
    a, k1 = _ptr(f, n * q)
    b, k2 = _ptr(g, n * q)
    _check(lib, lib.lbm_set_populations(ctx, a, b, _one_kind(k1, k2)), ctx)


def lbm_diag(ctx, phase_eps: float = 1e-3) -> dict:
    lib = load()
    out = LbmDiagOut()
    code = lib.lbm_diag(ctx, float(phase_eps), ctypes.byref(out))
    if code not in (LBM_OK, LBM_ERR_DIVERGED):
        _check(lib, code, ctx)
    return {k: getattr(out, k) for k, _ in LbmDiagOut._fields_ if k != "reserved"}


def lbm_diag_last(ctx):
    """(record, step) of the last in-step diagnostic of lbm_step (step -1 if none)."""
    lib = load()
    out = LbmDiagOut()
    step = ctypes.c_int64()
    _check(lib, lib.lbm_diag_last(ctx, ctypes.byref(out), ctypes.byref(step)), ctx)
    return {k: getattr(out, k) for k, _ in LbmDiagOut._fields_ if k != "reserved"}, step.value


def lbm_sync(ctx):
    lib = load()
    _check(lib, lib.lbm_sync(ctx), ctx)


def lbm_shape(ctx):
    lib = load()
    n, q = ctypes.c_int64(), ctypes.c_int32()
    _check(lib, lib.lbm_shape(ctx, ctypes.byref(n), ctypes.byref(q)), ctx)
    return n.value, q.value


def lbm_last_error(ctx=None) -> str:
    msg = load().lbm_last_error(ctx)
    return msg.decode() if msg else ""


def lbm_destroy(ctx):
    lib = load()
    _check(lib, lib.lbm_destroy(ctx))


def lbm_advect_phase(ctx, u, scale: float = 1.0, nsteps: int = 1):
    lib = load()
    n, _, d = _dims(ctx)
    a, k = _ptr(u, n * d)
    _check(lib, lib.lbm_advect_phase(ctx, a, float(scale), int(nsteps), k), ctx)


def lbm_jet_stats(ctx, threshold: float = 0.5, max_drops: int = 4096) -> dict:
    """Breakup length and drops of the current state (see include/lbm.h)."""
    lib = load()
    out = LbmJetStats()
    vols = np.zeros(max(int(max_drops), 1), np.float64)
    _check(lib, lib.lbm_jet_stats(ctx, float(threshold), int(max_drops), vols.ctypes.data, ctypes.byref(out)), ctx)
    d = {k: getattr(out, k) for k, _ in LbmJetStats._fields_}
    d["drop_volumes"] = vols[:min(out.n_drops, int(max_drops))].copy()
    return d


def lbm_set_timing(ctx, enable: bool):
    lib = load()
    _check(lib, lib.lbm_set_timing(ctx, 1 if enable else 0), ctx)


def lbm_get_timing(ctx):
    """(ms_phi, ms_collide_stream, ms_faces, steps) summed since the last call."""
    lib = load()
    ms = (ctypes.c_double * 3)()
    n = ctypes.c_int64()
    _check(lib, lib.lbm_get_timing(ctx, ms, ctypes.byref(n)), ctx)
    return ms[0], ms[1], ms[2], n.value


def lbm_diag_noalloc(params: dict, f, g, phase_eps: float = 1e-3, stream=None) -> dict:
    """Diagnostics of device populations f, g ([Q][N] float32 CUDA tensors)
    without a context and without any device allocation (see include/lbm.h)."""
    lib = load()
    s = make_params(params)
    q = 9 if s.lattice == LBM_D2Q9 else 19
    n = q * s.nx * s.ny * s.nz
    pf, kf = _ptr(f, n)
    pg, kg = _ptr(g, n)
    if kf != 1 or kg != 1 or not (f.is_cuda and g.is_cuda):
        raise ValueError("lbm_diag_noalloc takes CUDA float32 tensors of Q * nx * ny * nz elements")
    out = LbmDiagOut()
    code = lib.lbm_diag_noalloc(ctypes.byref(s), pf, pg, float(phase_eps),
                                ctypes.byref(out), ctypes.c_void_p(_stream_handle(stream)))
    if code not in (LBM_OK, LBM_ERR_DIVERGED):
        _check(lib, code)
    return {k: getattr(out, k) for k, _ in LbmDiagOut._fields_ if k != "reserved"}


def lbm_collide_cells(params: dict, f, g, phin, fs, gs, out=None, stream=None):
    """Device tensors [n][Q] (out: [n][5]); see include/lbm.h."""
    lib = load()
    s = make_params(params)
    n = f.shape[0]
    ptrs = [_ptr(t)[0] for t in (f, g, phin, fs, gs)]
    o = _ptr(out)[0] if out is not None else None
    _check(lib, lib.lbm_collide_cells(ctypes.byref(s), int(n), *ptrs, o,
                                      ctypes.c_void_p(_stream_handle(stream))))


def _stream_handle(stream):
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ------------------------------------------------------------ convenience

class LBM:
    """One simulation context (grid + parameters + device state)."""

    def __init__(self, params: dict, stream=None):
        self.params = dict(params)
        self.lattice = int(params["lattice"])
        self.D = 2 if self.lattice == LBM_D2Q9 else 3
        self.Q = 9 if self.lattice == LBM_D2Q9 else 19
        self.shape = (int(params.get("nz", 1)), int(params["ny"]), int(params["nx"]))
        self.N = int(np.prod(self.shape))
        self._h = lbm_create(params, stream)

    def close(self):
        if getattr(self, "_h", None):
            lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, phi, u=None, pstar=None):
        if not _is_torch(phi):
            phi = np.ascontiguousarray(phi, np.float32)
            u = None if u is None else np.ascontiguousarray(u, np.float32)
            pstar = None if pstar is None else np.ascontiguousarray(pstar, np.float32)
        lbm_init_fields(self._h, phi, u, pstar, n=self.N, dim=self.D)

    def step(self, n: int = 1):
        lbm_step(self._h, n)

    def sync(self):
        lbm_sync(self._h)

    def diag_last(self):
        return lbm_diag_last(self._h)

    def fields(self):
        phi = np.empty(self.shape, np.float32)
        u = np.empty((self.D,) + self.shape, np.float32)
        p = np.empty(self.shape, np.float32)
        lbm_get_fields(self._h, phi, u, p)
        return phi, u, p

    def populations(self):
        f = np.empty((self.Q,) + self.shape, np.float32)
        g = np.empty((self.Q,) + self.shape, np.float32)
        lbm_get_populations(self._h, f, g)
        return f, g

    def set_populations(self, f, g):
        if not _is_torch(f):
            f = np.ascontiguousarray(f, np.float32)
            g = np.ascontiguousarray(g, np.float32)
        lbm_set_populations(self._h, f, g)

    def diag(self, phase_eps: float = 1e-3) -> dict:
        return lbm_diag(self._h, phase_eps)

    def jet_stats(self, threshold: float = 0.5, max_drops: int = 4096) -> dict:
        return lbm_jet_stats(self._h, threshold, max_drops)

    def advect(self, u, scale: float = 1.0, nsteps: int = 1):
        """Advance only the phase field in the velocity scale * u (see lbm_advect_phase)."""
        if not _is_torch(u):
            u = np.ascontiguousarray(u, np.float32)
        lbm_advect_phase(self._h, u, scale, nsteps)

    def set_timing(self, enable: bool = True):
        lbm_set_timing(self._h, enable)

    def timing(self):
        return lbm_get_timing(self._h)


# ------------------------------------------------------------ batched sweeps

def _bcheck(lib, code, b=None):
    if code != LBM_OK:
        msg = lib.lbm_batch_last_error(b)
        raise LbmError(code, msg.decode() if msg else "")


def lbm_batch_create(params_list, stream=None):
    lib = load()
    arr = (LbmParams * len(params_list))(*[make_params(p) for p in params_list])
    h = ctypes.c_void_p()
    _bcheck(lib, lib.lbm_batch_create(arr, len(params_list), ctypes.c_void_p(_stream_handle(stream)),
                                      ctypes.byref(h)))
    return h


def lbm_batch_init_fields(b, c: int, phi, u=None, pstar=None):
    lib = load()
    a, k1 = _ptr(phi)
    v, k2 = _ptr(u)
    w, k3 = _ptr(pstar)
    _bcheck(lib, lib.lbm_batch_init_fields(b, int(c), a, v, w, _one_kind(k1, k2, k3)), b)


def lbm_batch_step(b, nsteps: int):
    lib = load()
    _bcheck(lib, lib.lbm_batch_step(b, int(nsteps)), b)


def lbm_batch_get_fields(b, c: int, phi=None, u=None, p=None):
    lib = load()
    a, k1 = _ptr(phi)
    v, k2 = _ptr(u)
    w, k3 = _ptr(p)
    _bcheck(lib, lib.lbm_batch_get_fields(b, int(c), a, v, w, _one_kind(k1, k2, k3)), b)


def lbm_batch_diag(b, c: int, phase_eps: float = 1e-3) -> dict:
    lib = load()
    out = LbmDiagOut()
    code = lib.lbm_batch_diag(b, int(c), float(phase_eps), ctypes.byref(out))
    if code not in (LBM_OK, LBM_ERR_DIVERGED):
        _bcheck(lib, code, b)
    return {k: getattr(out, k) for k, _ in LbmDiagOut._fields_ if k != "reserved"}


def _plan_dict(pl: LbmBatchPlan) -> dict:
    n = pl.nclasses
    d = {"nclasses": n}
    for k in ("nx_max", "ncases", "tile_x", "seglen", "blocks_per_sm", "ms_per_step"):
        d[k] = list(getattr(pl, k))[:n]
    return d


def lbm_batch_get_plan(b) -> dict:
    lib = load()
    pl = LbmBatchPlan()
    _bcheck(lib, lib.lbm_batch_get_plan(b, ctypes.byref(pl)), b)
    return _plan_dict(pl)


def lbm_batch_set_plan(b, plan: dict):
    lib = load()
    pl = LbmBatchPlan()
    pl.nclasses = int(plan["nclasses"])
    for k in ("nx_max", "ncases", "tile_x", "seglen", "blocks_per_sm"):
        for i, v in enumerate(plan[k]):
            getattr(pl, k)[i] = int(v)
    _bcheck(lib, lib.lbm_batch_set_plan(b, ctypes.byref(pl)), b)


def lbm_batch_tune(b, trial_steps: int = 5) -> dict:
    lib = load()
    pl = LbmBatchPlan()
    _bcheck(lib, lib.lbm_batch_tune(b, int(trial_steps), ctypes.byref(pl)), b)
    return _plan_dict(pl)


def lbm_batch_sync(b):
    lib = load()
    _bcheck(lib, lib.lbm_batch_sync(b), b)


def lbm_batch_last_error(b=None) -> str:
    msg = load().lbm_batch_last_error(b)
    return msg.decode() if msg else ""


def lbm_batch_destroy(b):
    lib = load()
    _bcheck(lib, lib.lbm_batch_destroy(b))


class Batch:
    """Many independent cases advanced together (see include/lbm.h)."""

    def __init__(self, params_list, stream=None):
        self.params = [dict(p) for p in params_list]
        self.D = 2 if not self.params or int(self.params[0]["lattice"]) == LBM_D2Q9 else 3
        self.shapes = [(int(p.get("nz", 1)), int(p["ny"]), int(p["nx"])) for p in self.params]
        self._h = lbm_batch_create(self.params, stream)

    def close(self):
        if getattr(self, "_h", None):
            lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.params)

    def init_fields(self, c, phi, u=None, pstar=None):
        if not _is_torch(phi):
            phi = np.ascontiguousarray(phi, np.float32)
            u = None if u is None else np.ascontiguousarray(u, np.float32)
            pstar = None if pstar is None else np.ascontiguousarray(pstar, np.float32)
        lbm_batch_init_fields(self._h, c, phi, u, pstar)

    def step(self, n: int = 1):
        lbm_batch_step(self._h, n)

    def sync(self):
        lbm_batch_sync(self._h)

    def fields(self, c):
        sh = self.shapes[c]
        phi = np.empty(sh, np.float32)
        u = np.empty((self.D,) + sh, np.float32)
        p = np.empty(sh, np.float32)
        lbm_batch_get_fields(self._h, c, phi, u, p)
        return phi, u, p

    def diag(self, c, phase_eps: float = 1e-3) -> dict:
        return lbm_batch_diag(self._h, c, phase_eps)

    def plan(self) -> dict:
        return lbm_batch_get_plan(self._h)

    def set_plan(self, plan: dict):
        lbm_batch_set_plan(self._h, plan)

    def tune(self, trial_steps: int = 5) -> dict:
        return lbm_batch_tune(self._h, trial_steps)
