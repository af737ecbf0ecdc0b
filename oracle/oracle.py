"""ctypes binding of the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module.  The product library never
imports it.  It shares no code with the CUDA path.

Conventions: arrays are numpy, fields are ``[nz][ny][nx]`` (x fastest), the
velocity is ``D`` consecutive planes, populations are population-major
``[Q][nz][ny][nx]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liblbm_oracle.so")
# a prebuilt oracle library may be substituted (the mutation tests use this)
LIB_OVERRIDE = os.environ.get("LBM_ORACLE_LIB")

D2Q9, D3Q19 = 0, 1
PERIODIC, WALL, INLET, OUTFLOW = 0, 1, 2, 3


def compile_source(src: str, out: str) -> str:
    """gcc -O2 with FP contraction off (so x86 and Arm agree), OpenMP if available."""
    tmp = out + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", src, "-o", tmp, "-lm"]
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:])
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build (skipped when up to date)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    return compile_source(SRC, LIB)


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 6),
        ("visc_model", ctypes.c_int32), ("outlet_scheme", ctypes.c_int32),
        ("rho_L", ctypes.c_double), ("rho_H", ctypes.c_double),
        ("tau_L", ctypes.c_double), ("tau_H", ctypes.c_double),
        ("mu_ratio", ctypes.c_double),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double),
        ("mobility", ctypes.c_double),
        ("force", ctypes.c_double * 3), ("rho_ref", ctypes.c_double),
        ("inlet_u", ctypes.c_double),
        ("inlet_center", ctypes.c_double * 2),
        ("inlet_radius", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(LIB_OVERRIDE if LIB_OVERRIDE else build())
        d = ctypes.POINTER(ctypes.c_double)
        f = ctypes.POINTER(ctypes.c_float)
        i32 = ctypes.POINTER(ctypes.c_int32)
        _lib.orc_create.restype = ctypes.c_void_p
        _lib.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
        _lib.orc_validate.argtypes = [ctypes.POINTER(OrcParams)]
        _lib.orc_destroy.argtypes = [ctypes.c_void_p]
        _lib.orc_init.argtypes = [ctypes.c_void_p, f, f, f]
        _lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        _lib.orc_fields.argtypes = [ctypes.c_void_p, d, d, d]
        _lib.orc_get_pops.argtypes = [ctypes.c_void_p, d, d]
        _lib.orc_set_pops.argtypes = [ctypes.c_void_p, d, d]
        _lib.orc_lattice.argtypes = [ctypes.c_int, i32, d, i32]
        _lib.orc_matrix.argtypes = [ctypes.c_int, d]
        _lib.orc_collision_matrix.argtypes = [ctypes.c_int, ctypes.c_double, d]
        _lib.orc_collide_node.argtypes = [ctypes.c_void_p, d, d, d, d, d, d, d]
        _lib.orc_advect.argtypes = [ctypes.c_void_p, d, ctypes.c_double, ctypes.c_int64]
        _lib.orc_advect.restype = ctypes.c_int
        _lib.orc_apply_faces.argtypes = [ctypes.c_void_p, d, d]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if a is not None else None


def lattice(lat: int):
    e = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    Q = lib().orc_lattice(lat, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(w),
                          opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return e[:Q].copy(), w[:Q].copy(), opp[:Q].copy()


def matrix(lat: int) -> np.ndarray:
    Q = 9 if lat == D2Q9 else 19
    M = np.zeros(Q * Q)
    lib().orc_matrix(lat, _dp(M))
    return M.reshape(Q, Q)


def collision_matrix(lat: int, s_nu: float) -> np.ndarray:
    Q = 9 if lat == D2Q9 else 19
    C = np.zeros(Q * Q)
    if lib().orc_collision_matrix(lat, float(s_nu), _dp(C)) < 0:
        raise RuntimeError("singular transformation matrix")
    return C.reshape(Q, Q)


def make_params(p: dict) -> OrcParams:
    """Fill the oracle's parameter struct from a plain dict of case parameters."""
    s = OrcParams()
    s.lattice = int(p["lattice"])
    s.nx, s.ny, s.nz = int(p["nx"]), int(p["ny"]), int(p.get("nz", 1))
    for i, b in enumerate(p.get("bc", [PERIODIC] * 6)):
        s.bc[i] = int(b)
    s.visc_model = int(p.get("visc_model", 0))
    s.outlet_scheme = int(p.get("outlet_scheme", 0))
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
    return s


@dataclass
class Oracle:
    """One oracle context: a grid, its parameters and its FP64 state."""
    params: dict
    _h: int = field(default=0, init=False)

    def __post_init__(self):
        self._p = make_params(self.params)
        self.lat = self._p.lattice
        self.Q = 9 if self.lat == D2Q9 else 19
        self.D = 2 if self.lat == D2Q9 else 3
        self.shape = (self._p.nz, self._p.ny, self._p.nx)
        self.N = int(np.prod(self.shape))
        h = lib().orc_create(ctypes.byref(self._p))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = h

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, phi, u=None, pstar=None):
        phi = np.ascontiguousarray(phi, np.float32).reshape(-1)
        assert phi.size == self.N
        u = None if u is None else np.ascontiguousarray(u, np.float32).reshape(-1)
        if u is not None:
            assert u.size == self.D * self.N
        pstar = None if pstar is None else np.ascontiguousarray(pstar, np.float32).reshape(-1)
        lib().orc_init(self._h, _fp(phi), _fp(u), _fp(pstar))

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def fields(self):
        phi = np.zeros(self.N)
        u = np.zeros(self.D * self.N)
        p = np.zeros(self.N)
        lib().orc_fields(self._h, _dp(phi), _dp(u), _dp(p))
        return (phi.reshape(self.shape), u.reshape((self.D,) + self.shape),
                p.reshape(self.shape))

    def populations(self):
        f = np.zeros(self.Q * self.N)
        g = np.zeros(self.Q * self.N)
        lib().orc_get_pops(self._h, _dp(f), _dp(g))
        return f.reshape((self.Q,) + self.shape), g.reshape((self.Q,) + self.shape)

    def set_populations(self, f, g):
        f = np.ascontiguousarray(f, np.float64).reshape(-1)
        g = np.ascontiguousarray(g, np.float64).reshape(-1)
        assert f.size == self.Q * self.N and g.size == self.Q * self.N
        lib().orc_set_pops(self._h, _dp(f), _dp(g))

    def advect(self, u, scale=1.0, nsteps=1):
        """Advance only the phase field for nsteps in the velocity scale * u
        (u: D planes [nz][ny][nx]); see orc_advect."""
        ua = np.ascontiguousarray(u, np.float64).reshape(-1)
        if lib().orc_advect(self._h, _dp(ua), float(scale), int(nsteps)) != 0:
            raise ValueError("advection needs periodic or wall faces")

    def apply_faces(self, fB, gB):
        """The inlet and outlet rules of App. B applied to the post-streaming
        state (fB, gB) [Q][nz][ny][nx], with the current state as chi(N, t) of
        the outlet; returns the new arrays (see orc_apply_faces)."""
        fo = np.ascontiguousarray(fB, np.float64).reshape(-1).copy()
        go = np.ascontiguousarray(gB, np.float64).reshape(-1).copy()
        assert fo.size == self.Q * self.N and go.size == self.Q * self.N
        lib().orc_apply_faces(self._h, _dp(fo), _dp(go))
        return fo.reshape((self.Q,) + self.shape), go.reshape((self.Q,) + self.shape)

    def collide_node(self, f, g, phin):
        f = np.ascontiguousarray(f, np.float64)
        g = np.ascontiguousarray(g, np.float64)
        phin = np.ascontiguousarray(phin, np.float64)
        fs, gs, out, terms = np.zeros(self.Q), np.zeros(self.Q), np.zeros(5), np.zeros(15)
        lib().orc_collide_node(self._h, _dp(f), _dp(g), _dp(phin), _dp(fs), _dp(gs), _dp(out),
                               _dp(terms))
        names = ["phi", "gx", "gy", "gz", "lap", "rho", "tau", "mu_phi", "pstar",
                 "Fx", "Fy", "Fz", "ux", "uy", "uz"]
        return fs, gs, out, dict(zip(names, terms))


def threads() -> int:
    return int(lib().orc_threads())


def validate(params: dict) -> bool:
    s = make_params(params)
    return lib().orc_validate(ctypes.byref(s)) == 0
