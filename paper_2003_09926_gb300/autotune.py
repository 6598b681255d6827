"""Autotuner for the stage kernel's tile.

The FP32 vector-record stage kernel is built for three (i, j) tile shapes,
32 x 16, 16 x 32 and 16 x 16 nodes (the shared memory of a CTA is sized for
its tile: one CTA per SM for the first two, two for 16 x 16, the default),
and the third tile dimension, the number of
k-planes a CTA marches through (kc), is free.  Short chunks balance load
across SMs, long chunks amortise each chunk's prologue (four staged planes
and two node passes); a narrow tile wastes fewer padded columns on a grid
narrow in i, a small one on a small grid.  Both are chosen here by timing
candidates on scratch grids of the same shape (the caller's state is
untouched) with CUDA events; other precision modes have a fixed (i, j) tile
and only kc is tuned.  Results are cached per (precision, shape) for single
grids and per batch signature for batches, where one shape serves every grid.
"""
from __future__ import annotations

from . import jz

SHAPES = ((32, 16), (16, 32), (16, 16))
P32 = 2  # the precision mode whose default kernel has selectable tile shapes

_cache: dict = {}


def _time_ms(torch, fn, stream, reps: int) -> float:
    fn()  # warm-up (and graph capture)
    stream.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def candidates_for(nz: int) -> list[int]:
    out = sorted({c for c in (4, 8, 12, 16, 24, 32, 48, 64, 96, 128) if c < nz} | {nz})
    return out


def _nz(desc: dict) -> int:
    if desc["bc"][4] == 0:
        return desc["nk"] - 1 if desc.get("geom", 0) == 1 else desc["nk"]
    return desc["nk"] - 2


def _shapes(desc: dict):
    return SHAPES if desc.get("precision", 0) == P32 else (None,)


def apply(grid: jz.Grid, choice: dict) -> None:
    """Set a tuned choice {"shape": (ti, tj) or None, "kc": planes (0 = whole
    k range)} on a grid."""
    if choice.get("shape") is not None:
        jz.jz_set_tile_shape(grid.h, *choice["shape"])
    apply_kc(grid, choice["kc"])


def tune_grid(desc: dict, flow: dict, cfl: float = 0.5, reps: int = 3, device: int = 0) -> dict:
    """Best tile shape and k-chunk length for one grid of this shape and
    precision: {"shape": (ti, tj) or None, "kc": planes, "ms": step time}."""
    import torch
    key = ("grid", desc.get("precision", 0), desc.get("geom", 0), desc["ni"], desc["nj"], desc["nk"],
           tuple(desc["bc"]))
    if key in _cache:
        return _cache[key]
    stream = torch.cuda.Stream(device=device)
    g = jz.Grid(desc, stream=stream, device=device).init(flow, 0)
    best = {"shape": None, "kc": None, "ms": float("inf")}
    for shape in _shapes(desc):
        if shape is not None:
            jz.jz_set_tile_shape(g.h, *shape)
        for kc in candidates_for(_nz(desc)):
            jz.jz_set_tiling(g.h, kc)
            ms = _time_ms(torch, lambda: g.nsteps(1, cfl=cfl), stream, reps)
            if ms < best["ms"]:
                best = {"shape": shape, "kc": kc, "ms": ms}
    g.close()
    _cache[key] = best
    return best


def tune_batch(cases: list[tuple[dict, dict]], cfl: float = 0.5, reps: int = 2, device: int = 0,
               candidates=(4, 8, 16, 32, 64, 0)) -> dict:
    """Best tile shape and uniform k-chunk length (0 = whole k range) for a
    batch of grids (list of (grid desc, flow)), timed with batched steps on
    scratch grids: {"shape": (ti, tj) or None, "kc": planes, "ms": step time}."""
    import torch
    sig = ("batch",) + tuple(sorted((d.get("precision", 0), d.get("geom", 0), d["ni"], d["nj"], d["nk"])
                                    for d, _ in cases))
    if sig in _cache:
        return _cache[sig]
    stream = torch.cuda.Stream(device=device)
    grids = [jz.Grid(d, stream=stream, device=device).init(f, 0) for d, f in cases]
    best = {"shape": None, "kc": None, "ms": float("inf")}
    for shape in _shapes(cases[0][0]):
        for kc in candidates:
            for g in grids:
                apply(g, {"shape": shape, "kc": kc})
            b = jz.Batch(grids, stream=stream)
            ms = _time_ms(torch, lambda: b.nsteps(1, cfl), stream, reps)
            b.close()
            if ms < best["ms"]:
                best = {"shape": shape, "kc": kc, "ms": ms}
    for g in grids:
        g.close()
    _cache[sig] = best
    return best


def apply_kc(grid: jz.Grid, kc: int) -> None:
    nz = _nz(grid.desc)
    jz.jz_set_tiling(grid.h, nz if kc == 0 else min(kc, nz))
