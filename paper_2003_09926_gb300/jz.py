"""Thin Python binding of the C ABI in ``include/jz.h`` (argument marshalling
only; every step of the method runs in the CUDA kernels of ``libjz.so``).

The module-level functions carry the C names (``jz_grid_bytes``,
``jz_grid_create``, ...).  ``Grid`` and ``Batch`` are small conveniences on
top of them: they allocate the caller-owned device buffer with PyTorch and
pass a CUDA stream handle.  Importing this module never falls back to a CPU
path: if ``libjz.so`` is missing or fails to load, it raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjz.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "jz.h")

JZ_OK, JZ_EINVAL, JZ_ENOMEM, JZ_ECUDA, JZ_ENONFINITE, JZ_ETIMEOUT = 0, -1, -2, -3, -4, -5
ERRNAMES = {-1: "JZ_EINVAL", -2: "JZ_ENOMEM", -3: "JZ_ECUDA", -4: "JZ_ENONFINITE", -5: "JZ_ETIMEOUT"}


class JzError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("ni", C.c_int), ("nj", C.c_int), ("nk", C.c_int), ("bc", C.c_int * 6),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("cluster_r", C.c_double), ("stretch_c", C.c_double), ("stretch_w", C.c_double),
                ("map_amp", C.c_double), ("map_seed", C.c_uint64), ("precision", C.c_int), ("geom", C.c_int)]


class FlowParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("mach", "re", "gamma", "pr", "prt", "cs", "k2", "k4", "sigma", "s1", "r0", "theta", "noise")] + [
        ("ic", C.c_int), ("sgs", C.c_int)]


class Diag(C.Structure):
    _fields_ = [("time", C.c_double), ("step", C.c_int64), ("dt", C.c_double), ("sum", C.c_double * 5),
                ("rho_min", C.c_double), ("rho_max", C.c_double), ("p_min", C.c_double), ("p_max", C.c_double),
                ("mach_max", C.c_double), ("nonfinite", C.c_int64)]


_lib = None


def lib() -> C.CDLL:
    """Load ``libjz.so`` (built in-tree by ``build.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        P, VP, G, B = C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p
        sig = {
            "jz_last_error": ([C.c_char_p, C.c_size_t], C.c_int),
            "jz_grid_bytes": ([C.POINTER(GridDesc), C.POINTER(C.c_size_t)], C.c_int),
            "jz_grid_create": ([C.POINTER(GridDesc), VP, C.c_size_t, VP, C.POINTER(G)], C.c_int),
            "jz_grid_destroy": ([G], C.c_int),
            "jz_state_init": ([G, C.POINTER(FlowParams), C.c_uint64], C.c_int),
            "jz_rk_step": ([G, C.c_double, C.c_double], C.c_int),
            "jz_nsteps": ([G, C.c_int, C.c_double, C.c_double], C.c_int),
            "jz_diagnostics": ([G, C.POINTER(Diag)], C.c_int),
            "jz_diagnostics_async": ([G, VP], C.c_int),
            "jz_set_step_diagnostics": ([G, C.c_int], C.c_int),
            "jz_step_diagnostics_async": ([G, VP], C.c_int),
            "jz_state_download": ([G, C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "jz_state_upload": ([G, C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "jz_metrics_download": ([G, C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "jz_batch_bytes": ([C.POINTER(G), C.c_int, C.POINTER(C.c_size_t)], C.c_int),
            "jz_batch_create": ([C.POINTER(G), C.c_int, VP, C.c_size_t, VP, C.POINTER(B)], C.c_int),
            "jz_batch_nsteps": ([B, C.c_int, C.c_double], C.c_int),
            "jz_batch_destroy": ([B], C.c_int),
            "jz_block_bytes": ([C.POINTER(GridDesc), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)],
                               C.c_int),
            "jz_block_create": ([C.POINTER(GridDesc), C.POINTER(C.c_int), C.POINTER(C.c_int), VP, C.c_size_t, VP,
                                 C.POINTER(G)], C.c_int),
            "jz_blocks_bytes": ([C.POINTER(G), C.c_int, C.POINTER(C.c_size_t)], C.c_int),
            "jz_stats_bytes": ([G, C.POINTER(C.c_size_t)], C.c_int),
            "jz_stats_create": ([G, VP, C.c_size_t, C.POINTER(VP)], C.c_int),
            "jz_stats_sample": ([VP], C.c_int),
            "jz_stats_count": ([VP, C.POINTER(C.c_int64)], C.c_int),
            "jz_stats_read": ([VP, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_size_t], C.c_int),
            "jz_stats_radial": ([VP, C.c_double, C.c_int, C.c_double, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
            "jz_stats_core_length": ([VP, C.c_double, C.c_double, C.POINTER(C.c_double)], C.c_int),
            "jz_stats_destroy": ([VP], C.c_int),
            "jz_set_clock": ([G, C.c_double, C.c_int64], C.c_int),
            "jz_blocks_create": ([C.POINTER(G), C.c_int, VP, C.c_size_t, VP, C.POINTER(B)], C.c_int),
            "jz_launch_count": ([C.POINTER(C.c_uint64)], C.c_int),
            "jz_profile_begin": ([G], C.c_int),
            "jz_profile_read": ([G, C.POINTER(C.c_double), C.POINTER(C.c_int64)], C.c_int),
            "jz_profile_end": ([G], C.c_int),
            "jz_get_tiling": ([G, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
            "jz_set_tiling": ([G, C.c_int], C.c_int),
            "jz_set_stage_variant": ([G, C.c_int], C.c_int),
            "jz_set_stall_test": ([G, C.c_int], C.c_int),
            "jz_set_stream": ([G, VP], C.c_int),
            "jz_halo_bytes": ([G, C.c_int, C.POINTER(C.c_size_t)], C.c_int),
            "jz_halo_pack": ([G, C.c_int, C.c_int, C.c_int, VP], C.c_int),
            "jz_halo_unpack": ([G, C.c_int, C.c_int, C.c_int, VP], C.c_int),
            "jz_block_rate": ([G, C.POINTER(C.c_void_p)], C.c_int),
            "jz_block_advance": ([G, C.c_double], C.c_int),
            "jz_block_stage": ([G, C.c_int], C.c_int),
            "jz_set_tile_shape": ([G, C.c_int, C.c_int], C.c_int),
            "jz_fma_peak": ([C.c_int, C.POINTER(C.c_double), VP], C.c_int),
        }
        sig["jz_state_diagnostics_static"] = ([C.c_longlong, C.c_int, VP, VP, C.c_double, VP, VP], C.c_int)
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes, f.restype = args, res
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of every function declared in include/jz.h."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\bint\s+(jz_\w+)\s*\(", text)))


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    lib().jz_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


def _check(rc: int) -> int:
    if rc != JZ_OK:
        raise JzError(rc, last_error())
    return rc


def make_desc(d: dict) -> GridDesc:
    g = GridDesc()
    g.ni, g.nj, g.nk = d["ni"], d["nj"], d["nk"]
    for f in range(6):
        g.bc[f] = d["bc"][f]
    for a in range(3):
        g.lo[a], g.hi[a] = d["lo"][a], d["hi"][a]
    g.cluster_r = d.get("cluster_r", 0.5)
    g.stretch_c = d.get("stretch_c", 0.0)
    g.stretch_w = d.get("stretch_w", 0.5)
    g.map_amp = d.get("map_amp", 0.0)
    g.map_seed = d.get("map_seed", 0)
    g.precision = d.get("precision", 0)
    g.geom = d.get("geom", 0)
    return g


def make_flow(f: dict) -> FlowParams:
    p = FlowParams()
    for n, _ in FlowParams._fields_:
        setattr(p, n, f.get(n, 0) if n == "sgs" else f[n])
    return p


# ---- C-named entry points ---------------------------------------------------

def jz_grid_bytes(desc: dict) -> int:
    out = C.c_size_t(0)
    _check(lib().jz_grid_bytes(C.byref(make_desc(desc)), C.byref(out)))
    return out.value


def jz_grid_create(desc: dict, dev_ptr: int, nbytes: int, stream: int) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().jz_grid_create(C.byref(make_desc(desc)), C.c_void_p(dev_ptr), nbytes, C.c_void_p(stream), C.byref(h)))
    return h


def jz_block_bytes(desc: dict, o0, o1) -> int:
    out = C.c_size_t(0)
    a, b = (C.c_int * 3)(*o0), (C.c_int * 3)(*o1)
    _check(lib().jz_block_bytes(C.byref(make_desc(desc)), a, b, C.byref(out)))
    return out.value


def jz_block_create(desc: dict, o0, o1, dev_ptr: int, nbytes: int, stream: int) -> C.c_void_p:
    h = C.c_void_p()
    a, b = (C.c_int * 3)(*o0), (C.c_int * 3)(*o1)
    _check(lib().jz_block_create(C.byref(make_desc(desc)), a, b, C.c_void_p(dev_ptr), nbytes, C.c_void_p(stream),
                                 C.byref(h)))
    return h


def jz_grid_destroy(h) -> None:
    _check(lib().jz_grid_destroy(h))


def jz_state_init(h, flow: dict, seed: int) -> None:
    _check(lib().jz_state_init(h, C.byref(make_flow(flow)), C.c_uint64(seed)))


def jz_rk_step(h, cfl: float = 0.0, dt_fixed: float = 0.0) -> None:
    _check(lib().jz_rk_step(h, cfl, dt_fixed))


def jz_nsteps(h, n: int, cfl: float = 0.0, dt_fixed: float = 0.0) -> None:
    _check(lib().jz_nsteps(h, n, cfl, dt_fixed))


def jz_diagnostics(h, allow_nonfinite: bool = False) -> dict:
    d = Diag()
    rc = lib().jz_diagnostics(h, C.byref(d))
    if rc != JZ_OK and not (allow_nonfinite and rc == JZ_ENONFINITE):
        raise JzError(rc, last_error())
    return {"time": d.time, "step": d.step, "dt": d.dt, "sum": np.array(list(d.sum)), "rho_min": d.rho_min,
            "rho_max": d.rho_max, "p_min": d.p_min, "p_max": d.p_max, "mach_max": d.mach_max,
            "nonfinite": d.nonfinite, "status": rc}


def diag_dict(d: Diag) -> dict:
    return {"time": d.time, "step": d.step, "dt": d.dt, "sum": np.array(list(d.sum)), "rho_min": d.rho_min,
            "rho_max": d.rho_max, "p_min": d.p_min, "p_max": d.p_max, "mach_max": d.mach_max,
            "nonfinite": d.nonfinite}


class PinnedDiag:
    """A jz_diag record in page-locked host memory (a pinned torch tensor), the
    target of Grid.diagnostics_async and Grid.step_diagnostics_async."""

    def __init__(self):
        torch = _torch()
        self._buf = torch.zeros(C.sizeof(Diag), dtype=torch.uint8, pin_memory=True)
        self.ptr = self._buf.data_ptr()

    def read(self) -> dict:
        """The record as a dict (valid once the stream has passed the copy)."""
        return diag_dict(Diag.from_address(self.ptr))


def jz_state_download(h, out: np.ndarray) -> np.ndarray:
    assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
    _check(lib().jz_state_download(h, out.ctypes.data_as(C.POINTER(C.c_double)), out.size))
    return out


def jz_metrics_download(h, out: np.ndarray) -> np.ndarray:
    assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
    _check(lib().jz_metrics_download(h, out.ctypes.data_as(C.POINTER(C.c_double)), out.size))
    return out


def jz_state_upload(h, Q: np.ndarray) -> None:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    _check(lib().jz_state_upload(h, Q.ctypes.data_as(C.POINTER(C.c_double)), Q.size))


def jz_launch_count() -> int:
    out = C.c_uint64(0)
    _check(lib().jz_launch_count(C.byref(out)))
    return out.value


def jz_profile_begin(h) -> None:
    _check(lib().jz_profile_begin(h))


def jz_profile_read(h):
    ms = (C.c_double * 4)()
    n = (C.c_int64 * 4)()
    _check(lib().jz_profile_read(h, ms, n))
    return list(ms), list(n)


def jz_profile_end(h) -> None:
    _check(lib().jz_profile_end(h))


def jz_get_tiling(h):
    ti, tj, kc = C.c_int(), C.c_int(), C.c_int()
    _check(lib().jz_get_tiling(h, C.byref(ti), C.byref(tj), C.byref(kc)))
    return ti.value, tj.value, kc.value


def jz_set_tiling(h, kc: int) -> None:
    _check(lib().jz_set_tiling(h, kc))


def jz_set_stage_variant(h, variant: int) -> None:
    _check(lib().jz_set_stage_variant(h, variant))


def jz_halo_bytes(h, d: int) -> int:
    n = C.c_size_t()
    _check(lib().jz_halo_bytes(h, d, C.byref(n)))
    return n.value


def jz_halo_pack(h, which: int, d: int, side: int, dev_ptr: int) -> None:
    _check(lib().jz_halo_pack(h, which, d, side, C.c_void_p(dev_ptr)))


def jz_halo_unpack(h, which: int, d: int, side: int, dev_ptr: int) -> None:
    _check(lib().jz_halo_unpack(h, which, d, side, C.c_void_p(dev_ptr)))


def jz_block_rate(h) -> int:
    """Enqueue the block's rate; returns the device address of its FP64 scalar."""
    p = C.c_void_p()
    _check(lib().jz_block_rate(h, C.byref(p)))
    return p.value


def jz_block_advance(h, cfl: float) -> None:
    _check(lib().jz_block_advance(h, cfl))


def jz_block_stage(h, stage: int) -> None:
    _check(lib().jz_block_stage(h, stage))


def jz_set_stall_test(h, on: bool) -> None:
    _check(lib().jz_set_stall_test(h, int(bool(on))))


def jz_set_tile_shape(h, ti: int, tj: int) -> None:
    _check(lib().jz_set_tile_shape(h, ti, tj))


def jz_fma_peak(fp64: bool, stream: int = 0) -> float:
    """Measured FMA throughput of the current device, TFLOP/s."""
    out = C.c_double(0.0)
    _check(lib().jz_fma_peak(1 if fp64 else 0, C.byref(out), C.c_void_p(stream)))
    return out.value


def jz_state_diagnostics_static(n_nodes: int, fp64: bool, q_ptr: int, vol_ptr: int, gamma: float, out_ptr: int,
                                stream: int) -> None:
    """Diagnostics of dense device arrays with no device allocation (the
    reduction scratch is a static device array inside the library)."""
    _check(lib().jz_state_diagnostics_static(n_nodes, 1 if fp64 else 0, C.c_void_p(q_ptr), C.c_void_p(vol_ptr),
                                             gamma, C.c_void_p(out_ptr), C.c_void_p(stream)))


# ---- conveniences -----------------------------------------------------------

def _torch():
    import torch  # device memory and streams only
    return torch


class Grid:
    """A grid living in a torch-allocated device buffer on a CUDA stream;
    with ``block=(o0, o1)`` the block of nodes [o0, o1] (i, j, k order,
    inclusive) of the grid ``desc`` describes."""

    def __init__(self, desc: dict, stream=None, device: int = 0, block=None):
        torch = _torch()
        self.desc = dict(desc)
        self.device = device
        self.block = None if block is None else (tuple(block[0]), tuple(block[1]))
        if self.block is None:
            self.nbytes = jz_grid_bytes(desc)
            ni, nj, nk = desc["ni"], desc["nj"], desc["nk"]
        else:
            self.nbytes = jz_block_bytes(desc, *self.block)
            ni, nj, nk = (self.block[1][a] - self.block[0][a] + 1 for a in range(3))
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=f"cuda:{device}")
        ptr = self.buf.data_ptr()
        self.ptr = (ptr + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        if self.block is None:
            self.h = jz_grid_create(desc, self.ptr, self.nbytes, self.stream.cuda_stream)
        else:
            self.h = jz_block_create(desc, *self.block, self.ptr, self.nbytes, self.stream.cuda_stream)
        self.shape = (5, nk, nj, ni)

    def init(self, flow: dict, seed: int):
        self.flow = dict(flow)
        jz_state_init(self.h, flow, seed)
        return self

    def step(self, cfl: float = 0.0, dt: float = 0.0):
        jz_rk_step(self.h, cfl, dt)

    def nsteps(self, n: int, cfl: float = 0.0, dt: float = 0.0):
        jz_nsteps(self.h, n, cfl, dt)

    def diagnostics(self, allow_nonfinite: bool = False) -> dict:
        return jz_diagnostics(self.h, allow_nonfinite)

    def diagnostics_async(self, out: "PinnedDiag") -> None:
        """Enqueue the diagnostics and their copy into out on the grid's
        stream (no synchronisation; read out after the stream passes it)."""
        _check(lib().jz_diagnostics_async(self.h, C.c_void_p(out.ptr)))

    def set_step_diagnostics(self, on: bool) -> None:
        """Let every later CFL step's time-step reduction also form the
        diagnostics of the state the step starts from."""
        _check(lib().jz_set_step_diagnostics(self.h, int(bool(on))))

    def step_diagnostics_async(self, out: "PinnedDiag") -> None:
        """Enqueue the copy of the latest diagnostics record (after a step
        with step diagnostics on: the state that step started from) into
        out, without a pass over the grid."""
        _check(lib().jz_step_diagnostics_async(self.h, C.c_void_p(out.ptr)))

    def download(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shape)
        return jz_state_download(self.h, out)

    def set_stream(self, stream) -> None:
        """Enqueue later work on `stream` (a torch.cuda.Stream), after the work so far."""
        _check(lib().jz_set_stream(self.h, C.c_void_p(stream.cuda_stream)))
        self.stream = stream

    def metrics(self) -> np.ndarray:
        """[10][nk][nj][ni] FP64: S^k_m at 3k+m, J at 9."""
        return jz_metrics_download(self.h, np.empty((10,) + tuple(self.shape[1:])))

    def upload(self, Q: np.ndarray):
        assert Q.shape == self.shape
        jz_state_upload(self.h, Q)

    def synchronize(self):
        self.stream.synchronize()

    def save(self, path: str):
        """Restart file: the state of the grid's nodes (FP64) and its clock."""
        d = self.diagnostics(allow_nonfinite=True)
        np.savez(path, Q=self.download(), time=d["time"], step=d["step"], dt=d["dt"])

    def load(self, path: str):
        """Restart from a file written by save (the flow parameters are set by init)."""
        with np.load(path) as z:
            self.upload(z["Q"])
            _check(lib().jz_set_clock(self.h, float(z["time"]), int(z["step"])))
        return self

    def close(self):
        if getattr(self, "h", None):
            jz_grid_destroy(self.h)
            self.h = None
        self.buf = None  # return the device memory to the caller's allocator

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent grids stepped together; with ``coupled=True`` the blocks
    of one grid (halo exchange and one shared time step)."""

    def __init__(self, grids: list[Grid], stream=None, coupled: bool = False):
        torch = _torch()
        self.grids = grids
        arr = (C.c_void_p * len(grids))(*[g.h.value for g in grids])
        self._arr = arr
        nb = C.c_size_t(0)
        size_fn, create_fn = ((lib().jz_blocks_bytes, lib().jz_blocks_create) if coupled
                              else (lib().jz_batch_bytes, lib().jz_batch_create))
        _check(size_fn(arr, len(grids), C.byref(nb)))
        self.buf = torch.empty(nb.value + 256, dtype=torch.uint8, device=grids[0].buf.device)
        ptr = (self.buf.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.Stream(device=grids[0].device)
        self.h = C.c_void_p()
        _check(create_fn(arr, len(grids), C.c_void_p(ptr), nb.value, C.c_void_p(self.stream.cuda_stream),
                         C.byref(self.h)))

    def nsteps(self, n: int, cfl: float):
        _check(lib().jz_batch_nsteps(self.h, n, cfl))

    def close(self):
        if getattr(self, "h", None):
            lib().jz_batch_destroy(self.h)
            self.h = None
        self.buf = None


class Stats:
    """Time statistics of a grid's axial velocity (running sums on the device)."""

    def __init__(self, grid: Grid):
        torch = _torch()
        self.grid = grid
        nb = C.c_size_t(0)
        _check(lib().jz_stats_bytes(grid.h, C.byref(nb)))
        self.buf = torch.empty(nb.value + 256, dtype=torch.uint8, device=grid.buf.device)
        ptr = (self.buf.data_ptr() + 255) // 256 * 256
        self.h = C.c_void_p()
        _check(lib().jz_stats_create(grid.h, C.c_void_p(ptr), nb.value, C.byref(self.h)))

    def sample(self):
        _check(lib().jz_stats_sample(self.h))

    @property
    def samples(self) -> int:
        n = C.c_int64(0)
        _check(lib().jz_stats_count(self.h, C.byref(n)))
        return n.value

    def read(self):
        """(<U>, u_rms) per node, arrays of shape (nk, nj, ni)."""
        shape = self.grid.shape[1:]
        m, r = np.empty(shape), np.empty(shape)
        _check(lib().jz_stats_read(self.h, m.ctypes.data_as(C.POINTER(C.c_double)),
                                   r.ctypes.data_as(C.POINTER(C.c_double)), m.size))
        return m, r

    def radial(self, x: float, nbins: int, r_max: float):
        """(mean <U>, mean u_rms, node count) per radial bin at the plane nearest x."""
        m, r, c = np.empty(nbins), np.empty(nbins), np.empty(nbins)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        _check(lib().jz_stats_radial(self.h, x, nbins, r_max, dp(m), dp(r), dp(c)))
        return m, r, c

    def core_length(self, u_jet: float, frac: float = 0.95) -> float:
        out = C.c_double(0.0)
        _check(lib().jz_stats_core_length(self.h, u_jet, frac, C.byref(out)))
        return out.value

    def close(self):
        if getattr(self, "h", None):
            lib().jz_stats_destroy(self.h)
            self.h = None
        self.buf = None
