"""CPU FP64 oracle for the LES stage residual and 5-stage Runge-Kutta update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The GPU
product path (``paper_2003_09926_gb300``) never imports it and shares no code
with it.

The arithmetic lives in ``jz_oracle.c`` (plain C, double precision, one sweep
per step of the method, compiled with ``-ffp-contract=off``); this module only
builds it, marshals numpy arrays and offers a small object wrapper.  Every
function cites the passage of arXiv 2003.09926 it follows in the C source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jz_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NG = 2
BC_PERIODIC, BC_INFLOW, BC_FARFIELD = 0, 1, 2
IC_JET, IC_QUIESCENT = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP if present)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = base + ["-fopenmp", "-o", tmp, _SRC, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP runtime: build the single-threaded oracle
        cmd = base + ["-o", tmp, _SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [
        ("ni", C.c_int), ("nj", C.c_int), ("nk", C.c_int),
        ("bc", C.c_int * 6),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("cluster_r", C.c_double), ("stretch_c", C.c_double), ("stretch_w", C.c_double),
        ("map_amp", C.c_double), ("map_seed", C.c_uint64), ("geom", C.c_int),
    ]


class _Flow(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("mach", "re", "gamma", "pr", "prt", "cs", "k2", "k4", "sigma", "s1", "r0", "theta", "noise")] + [
        ("ic", C.c_int), ("sgs", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.POINTER(C.c_double)
            G, F = C.POINTER(_Grid), C.POINTER(_Flow)
            L.orc_npad.argtypes, L.orc_npad.restype = [G], C.c_size_t
            L.orc_splitmix64.argtypes, L.orc_splitmix64.restype = [C.c_uint64], C.c_uint64
            L.orc_map_params.argtypes = [G, C.POINTER(C.c_int), P]
            L.orc_base_coord.argtypes, L.orc_base_coord.restype = [G, C.c_int, C.c_double], C.c_double
            L.orc_coords.argtypes = [G, P]
            L.orc_metrics.argtypes = [G, P, P, P]
            L.orc_mu_inf.argtypes, L.orc_mu_inf.restype = [F], C.c_double
            L.orc_sutherland.argtypes, L.orc_sutherland.restype = [F, C.c_double], C.c_double
            L.orc_jet_profile.argtypes, L.orc_jet_profile.restype = [F, C.c_double], C.c_double
            L.orc_riemann_farfield.argtypes = [F, P, P, P]
            L.orc_apply_bc.argtypes = [G, F, P, P, P]
            L.orc_init.argtypes = [G, F, C.c_uint64, P, P, P]
            L.orc_residual.argtypes, L.orc_residual.restype = [G, F, P, P, P, P], C.c_int
            L.orc_max_rate.argtypes, L.orc_max_rate.restype = [G, F, P, P, P], C.c_double
            L.orc_rk_alpha.argtypes, L.orc_rk_alpha.restype = [C.c_int], C.c_double
            L.orc_rk_step.argtypes, L.orc_rk_step.restype = [G, F, P, P, P, P, C.c_double, C.c_double], C.c_double
            L.orc_diagnostics.argtypes = [G, F, P, P, P]
            L.orc_set_threads.argtypes, L.orc_set_threads.restype = [C.c_int], C.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_grid(desc: dict) -> _Grid:
    g = _Grid()
    g.ni, g.nj, g.nk = desc["ni"], desc["nj"], desc["nk"]
    for f in range(6):
        g.bc[f] = desc["bc"][f]
    for d in range(3):
        g.lo[d], g.hi[d] = desc["lo"][d], desc["hi"][d]
    g.cluster_r = desc.get("cluster_r", 0.5)
    g.stretch_c = desc.get("stretch_c", 0.0)
    g.stretch_w = desc.get("stretch_w", 0.5)
    g.map_amp = desc.get("map_amp", 0.0)
    g.map_seed = desc.get("map_seed", 0)
    g.geom = desc.get("geom", 0)
    return g


def make_flow(flow: dict) -> _Flow:
    f = _Flow()
    for n, _ in _Flow._fields_:
        setattr(f, n, flow.get(n, 0) if n == "sgs" else flow[n])
    return f


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def set_threads(n: int) -> int:
    return int(lib().orc_set_threads(n))


class Oracle:
    """One grid with its coordinates and metrics; state arrays are numpy
    (5, nk+4, nj+4, ni+4) float64 with two ghost layers on every face."""

    def __init__(self, desc: dict, flow: dict, X: np.ndarray | None = None):
        self.L = lib()
        self.desc, self.flowd = dict(desc), dict(flow)
        self.g = make_grid(desc)
        self.f = make_flow(flow)
        ni, nj, nk = desc["ni"], desc["nj"], desc["nk"]
        self.shape = (nk + 2 * NG, nj + 2 * NG, ni + 2 * NG)
        self.npad = int(self.L.orc_npad(C.byref(self.g)))
        assert self.npad == int(np.prod(self.shape))
        if X is None:
            X = np.zeros((3,) + self.shape)
            self.L.orc_coords(C.byref(self.g), _ptr(X))
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.S = np.zeros((9,) + self.shape)
        self.J = np.zeros(self.shape)
        self.L.orc_metrics(C.byref(self.g), _ptr(self.X), _ptr(self.S), _ptr(self.J))
        self.time, self.steps, self.last_dt = 0.0, 0, 0.0

    # views -----------------------------------------------------------------
    def inner(self, a: np.ndarray) -> np.ndarray:
        """Drop the ghost layers: (..., nk, nj, ni)."""
        return a[..., NG:-NG, NG:-NG, NG:-NG]

    def new_state(self) -> np.ndarray:
        return np.zeros((5,) + self.shape)

    # method ----------------------------------------------------------------
    def init(self, seed: int) -> np.ndarray:
        Q = self.new_state()
        self.L.orc_init(C.byref(self.g), C.byref(self.f), C.c_uint64(seed), _ptr(self.X), _ptr(self.S), _ptr(Q))
        return Q

    def apply_bc(self, Q: np.ndarray) -> np.ndarray:
        self.L.orc_apply_bc(C.byref(self.g), C.byref(self.f), _ptr(self.X), _ptr(self.S), _ptr(Q))
        return Q

    def residual(self, Q: np.ndarray) -> np.ndarray:
        R = self.new_state()
        if self.L.orc_residual(C.byref(self.g), C.byref(self.f), _ptr(self.S), _ptr(self.J), _ptr(Q), _ptr(R)):
            raise MemoryError("oracle residual: allocation failed")
        return R

    def max_rate(self, Q: np.ndarray) -> float:
        return float(self.L.orc_max_rate(C.byref(self.g), C.byref(self.f), _ptr(self.S), _ptr(self.J), _ptr(Q)))

    def step(self, Q: np.ndarray, cfl: float = 0.0, dt: float = 0.0) -> float:
        d = self.L.orc_rk_step(C.byref(self.g), C.byref(self.f), _ptr(self.X), _ptr(self.S), _ptr(self.J), _ptr(Q),
                               float(cfl), float(dt))
        if d < 0:
            raise MemoryError("oracle step: allocation failed")
        self.time += d
        self.steps += 1
        self.last_dt = d
        return d

    def run(self, Q: np.ndarray, n: int, cfl: float = 0.0, dt: float = 0.0) -> np.ndarray:
        for _ in range(n):
            self.step(Q, cfl, dt)
        return Q

    def diagnostics(self, Q: np.ndarray) -> dict:
        out = np.zeros(11)
        self.L.orc_diagnostics(C.byref(self.g), C.byref(self.f), _ptr(self.J), _ptr(Q), _ptr(out))
        return {"sum": out[0:5].copy(), "rho_min": out[5], "rho_max": out[6], "p_min": out[7], "p_max": out[8],
                "mach_max": out[9], "nonfinite": int(out[10])}

    # helpers for tests -------------------------------------------------------
    def sutherland(self, T: float) -> float:
        return float(self.L.orc_sutherland(C.byref(self.f), float(T)))

    def mu_inf(self) -> float:
        return float(self.L.orc_mu_inf(C.byref(self.f)))

    def riemann(self, qi, n) -> np.ndarray:
        qi = np.ascontiguousarray(qi, dtype=np.float64)
        n = np.ascontiguousarray(n, dtype=np.float64)
        qb = np.zeros(5)
        self.L.orc_riemann_farfield(C.byref(self.f), _ptr(qi), _ptr(n), _ptr(qb))
        return qb

    def map_params(self):
        m = (C.c_int * 9)()
        th = np.zeros(9)
        self.L.orc_map_params(C.byref(self.g), m, _ptr(th))
        return np.array(list(m)).reshape(3, 3), th.reshape(3, 3)

    def base_coord(self, d: int, idx: float) -> float:
        return float(self.L.orc_base_coord(C.byref(self.g), d, float(idx)))


def rk_alpha():
    return [lib().orc_rk_alpha(l) for l in range(5)]
