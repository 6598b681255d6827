"""Autotuner for the stage kernel's tile shape.

The (i, j) tile of the fused stage kernel is fixed per precision (32 x 16
nodes FP32, 16 x 16 FP64: one CTA per SM, shared memory sized for it); the
third tile dimension, the number of k-planes a CTA marches through (kc), is
chosen here by timing.  Short chunks balance load across SMs, long chunks
amortise each chunk's prologue (four staged planes and two node passes).
Candidates are timed on scratch grids of the same shape (the caller's state
is untouched) with CUDA events; results are cached per (precision, shape)
for single grids and per batch signature for batches.
"""
from __future__ import annotations

from . import jz

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


def tune_grid(desc: dict, flow: dict, cfl: float = 0.5, reps: int = 3, device: int = 0) -> int:
    """Best k-chunk length for one grid of this shape and precision."""
    import torch
    key = ("grid", desc.get("precision", 0), desc["ni"], desc["nj"], desc["nk"], tuple(desc["bc"]))
    if key in _cache:
        return _cache[key]
    stream = torch.cuda.Stream(device=device)
    g = jz.Grid(desc, stream=stream, device=device).init(flow, 0)
    nz = desc["nk"] if desc["bc"][4] == 0 else desc["nk"] - 2
    best, best_ms = None, float("inf")
    for kc in candidates_for(nz):
        jz.jz_set_tiling(g.h, kc)
        ms = _time_ms(torch, lambda: g.nsteps(1, cfl=cfl), stream, reps)
        if ms < best_ms:
            best, best_ms = kc, ms
    g.close()
    _cache[key] = best
    return best


def tune_batch(cases: list[tuple[dict, dict]], cfl: float = 0.5, reps: int = 2, device: int = 0,
               candidates=(4, 8, 16, 32, 64, 0)) -> int:
    """Best uniform k-chunk length (0 = whole k range) for a batch of grids
    (list of (grid desc, flow)), timed with batched steps on scratch grids."""
    import torch
    sig = ("batch",) + tuple(sorted((d.get("precision", 0), d["ni"], d["nj"], d["nk"]) for d, _ in cases))
    if sig in _cache:
        return _cache[sig]
    stream = torch.cuda.Stream(device=device)
    grids = [jz.Grid(d, stream=stream, device=device).init(f, 0) for d, f in cases]
    best, best_ms = None, float("inf")
    for kc in candidates:
        for g, (d, _) in zip(grids, cases):
            nz = d["nk"] if d["bc"][4] == 0 else d["nk"] - 2
            jz.jz_set_tiling(g.h, nz if kc == 0 else min(kc, nz))
        b = jz.Batch(grids, stream=stream)
        ms = _time_ms(torch, lambda: b.nsteps(1, cfl), stream, reps)
        b.close()
        if ms < best_ms:
            best, best_ms = kc, ms
    for g in grids:
        g.close()
    _cache[sig] = best
    return best


def apply_kc(grid: jz.Grid, kc: int) -> None:
    d = grid.desc
    nz = d["nk"] if d["bc"][4] == 0 else d["nk"] - 2
    jz.jz_set_tiling(grid.h, nz if kc == 0 else min(kc, nz))
