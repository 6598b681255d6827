"""Continuous-batching request loop for jet cases.

Requests (a grid, flow parameters, a seed, a step count and an arrival time)
are admitted in arrival order while their device footprint (``jz_grid_bytes``)
fits an HBM budget; admitted cases stay resident on the device and advance
together in time slices, each slice one batched launch sequence
(``jz_batch_nsteps``) over the resident grids it selects: all of them, or
(``fill_points``) cases in the order of ``order`` until they hold enough
points to fill the GPU -- "arrival" (oldest first) or "remaining" (least
remaining work, points x steps left, first: the smallest cases finish
first and share the GPU only where one case alone cannot fill it).
Finished cases are retired at slice boundaries -- their diagnostics (and
optionally their state) are read back and their memory returned -- so cases
that arrive while others run are admitted as soon as memory frees up and
their work overlaps on the device.  A request can be cancelled
(``Server.cancel``, or a ``cancel_at`` time in a trace): a waiting request
is dropped, a resident one is retired at the next slice boundary without a
result and its memory returned.  A case's result does not depend on the mix
it ran in: the per-point arithmetic of the batched kernels is that of a grid
stepped alone.

Latency of a case = completion - arrival (wall clock, seconds).
"""
from __future__ import annotations

import dataclasses
import threading
import time

import numpy as np

from . import jz
from . import workloads as W


@dataclasses.dataclass
class Request:
    rid: int
    grid: dict
    flow: dict
    seed: int
    steps: int
    arrival: float = 0.0
    cancel_at: float | None = None  # the client withdraws the request at this time (trace-driven)


@dataclasses.dataclass
class Result:
    rid: int
    status: str            # "done", "cancelled" or "rejected: <why>"
    arrival: float
    admitted: float = float("nan")
    finished: float = float("nan")
    points: int = 0
    steps: int = 0
    diag: dict | None = None
    state: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def updated_points(grid: dict) -> int:
    """Nodes the Runge-Kutta stages update (a cylinder's last azimuthal plane
    repeats its first)."""
    n = 1
    for a, key in enumerate(("ni", "nj", "nk")):
        if grid["bc"][2 * a] == W.BC_PERIODIC:
            n *= grid[key] - 1 if (a == 2 and grid.get("geom", W.GEOM_BOX) == W.GEOM_CYLINDER) else grid[key]
        else:
            n *= grid[key] - 2
    return n


def remaining_work(c: dict) -> int:
    """Point-steps a resident case still has to advance."""
    return updated_points(c["req"].grid) * c["left"]


def select_cases(resident: list[dict], fill_points: int | None, order: str = "arrival") -> list[dict]:
    """The resident cases one slice advances: every case when fill_points is
    None, else cases in the given order -- "arrival" (arrival, then id) or
    "remaining" (least remaining work, then arrival and id) -- until their
    updated points reach fill_points."""
    if fill_points is None:
        return list(resident)
    if order == "remaining":
        key = lambda c: (remaining_work(c), c["req"].arrival, c["req"].rid)  # noqa: E731
    elif order == "arrival":
        key = lambda c: (c["req"].arrival, c["req"].rid)  # noqa: E731
    else:
        raise ValueError(f"unknown order {order!r}")
    chosen, pts = [], 0
    for c in sorted(resident, key=key):
        chosen.append(c)
        pts += updated_points(c["req"].grid)
        if pts >= fill_points:
            break
    return chosen


class CudaBackend:
    """The device side of the server: grids and batches of the CUDA library
    on one stream (PyTorch supplies the stream only)."""

    def __init__(self, device: int = 0):
        import torch
        self.device = device
        self.stream = torch.cuda.Stream(device=device)

    def grid_bytes(self, desc: dict) -> int:
        return jz.jz_grid_bytes(desc)

    def grid(self, desc: dict, flow: dict, seed: int, kc: int | None):
        g = jz.Grid(desc, stream=self.stream, device=self.device).init(flow, seed)
        if kc is not None:
            jz.jz_set_tiling(g.h, int(kc))
        return g

    def batch(self, grids):
        return jz.Batch(grids, stream=self.stream)

    def synchronize(self):
        self.stream.synchronize()


class Server:
    def __init__(self, budget_bytes: int, slice_steps: int = 10, cfl: float = 0.5, device: int = 0,
                 keep_state: bool = False, kc_for=None, fill_points: int | None = None, order: str = "arrival",
                 backend=None):
        self.budget = int(budget_bytes)
        self.slice_steps = int(slice_steps)
        self.cfl = float(cfl)
        self.device = device
        self.keep_state = keep_state
        self.kc_for = kc_for  # optional callable grid-desc -> k-chunk length (autotuner)
        self.fill_points = fill_points
        if order not in ("arrival", "remaining"):
            raise ValueError(f"unknown order {order!r}")
        self.order = order
        self.backend = backend if backend is not None else CudaBackend(device)
        self.stream = getattr(self.backend, "stream", None)
        self.peak_bytes = 0
        self.slices = 0
        self._cancel_lock = threading.Lock()
        self._cancelled: set[int] = set()

    def cancel(self, rid: int) -> None:
        """Withdraw request rid (callable from another thread while run()
        executes): a waiting request is dropped; a resident one is retired at
        the next slice boundary, without a result, and its memory returned."""
        with self._cancel_lock:
            self._cancelled.add(int(rid))

    def run(self, requests: list[Request]) -> list[Result]:
        be = self.backend
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        results: dict[int, Result] = {}
        resident: list[dict] = []
        used = 0
        batches: dict = {}  # member ids -> Batch (its graph is kept while the members stay)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0

        def cancelled_now() -> set:
            t = now()
            with self._cancel_lock:
                out = set(self._cancelled)
            return out | {r.rid for r in requests if r.cancel_at is not None and r.cancel_at <= t}

        def drop_batches(live: set) -> None:
            for key in [k for k in batches if not set(k) <= live]:
                batches.pop(key).close()

        while pending or resident:
            # cancellations take effect here, between slices
            gone = cancelled_now()
            if gone:
                for r in [r for r in pending if r.rid in gone]:
                    pending.remove(r)
                    results[r.rid] = Result(r.rid, "cancelled", r.arrival, finished=now())
                hit = [c for c in resident if c["req"].rid in gone]
                if hit:
                    resident = [c for c in resident if c["req"].rid not in gone]
                    drop_batches({c["req"].rid for c in resident})
                    for c in hit:
                        res = results[c["req"].rid]
                        res.status, res.finished = "cancelled", now()
                        c["grid"].close()
                        used -= c["bytes"]
                if not pending and not resident:
                    break
            # admit in arrival order while the budget allows
            while pending and pending[0].arrival <= now():
                r = pending[0]
                need = be.grid_bytes(r.grid)
                if need > self.budget:
                    pending.pop(0)
                    results[r.rid] = Result(r.rid, f"rejected: needs {need} bytes, budget {self.budget}", r.arrival)
                    continue
                if used + need > self.budget:
                    break
                pending.pop(0)
                g = be.grid(r.grid, r.flow, r.seed, None if self.kc_for is None else self.kc_for(r.grid))
                used += need
                self.peak_bytes = max(self.peak_bytes, used)
                resident.append(dict(req=r, grid=g, left=r.steps, bytes=need))
                results[r.rid] = Result(r.rid, "running", r.arrival, admitted=now(), points=updated_points(r.grid),
                                        steps=r.steps)
            if not resident:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now())))
                continue
            chosen = select_cases(resident, self.fill_points, self.order)
            n = min(self.slice_steps, min(c["left"] for c in chosen))
            if len(chosen) == 1:  # one case: its own graph-replayed steps
                chosen[0]["grid"].nsteps(n, cfl=self.cfl)
            else:
                key = tuple(c["req"].rid for c in chosen)
                if key not in batches:
                    batches[key] = be.batch([c["grid"] for c in chosen])
                batches[key].nsteps(n, self.cfl)
            be.synchronize()
            self.slices += 1
            advanced = {id(c) for c in chosen}
            still = []
            for c in resident:
                if id(c) in advanced:
                    c["left"] -= n
                if c["left"] > 0:
                    still.append(c)
                    continue
                res = results[c["req"].rid]
                res.diag = c["grid"].diagnostics(allow_nonfinite=True)
                if self.keep_state:
                    res.state = c["grid"].download()
                res.finished = now()
                res.status = "done"
                c["grid"].close()
                used -= c["bytes"]
            if len(still) != len(resident):
                drop_batches({c["req"].rid for c in still})
                resident = still
        for b in batches.values():
            b.close()
        return [results[k] for k in sorted(results)]


def serve_one_at_a_time(requests: list[Request], precision: int, cfl: float = 0.5, device: int = 0,
                        keep_state: bool = False) -> list[Result]:
    """The plain baseline: requests in arrival order, one grid at a time, each
    run to completion with graph-replayed single-grid steps."""
    import torch
    stream = torch.cuda.Stream(device=device)
    out = []
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    for r in sorted(requests, key=lambda r: (r.arrival, r.rid)):
        while now() < r.arrival:
            time.sleep(min(0.01, r.arrival - now()))
        start = now()
        g = jz.Grid(dict(r.grid, precision=precision), stream=stream, device=device).init(r.flow, r.seed)
        g.nsteps(r.steps, cfl=cfl)
        stream.synchronize()
        res = Result(r.rid, "done", r.arrival, admitted=start, points=updated_points(r.grid), steps=r.steps)
        res.diag = g.diagnostics(allow_nonfinite=True)
        if keep_state:
            res.state = g.download()
        res.finished = now()
        g.close()
        out.append(res)
    return out


def summarize(results: list[Result]) -> dict:
    done = [r for r in results if r.status == "done"]
    if not done:
        return {"completed": 0}
    lat = np.array([r.latency for r in done])
    span = max(r.finished for r in done) - min(r.arrival for r in done)
    work = sum(r.points * 5 * r.steps for r in done)
    return {"completed": len(done), "rejected": len(results) - len(done),
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "makespan_s": float(span),
            "throughput_mpt_stage_s": work / span / 1e6 if span > 0 else None}


def poisson_trace(cfg: dict, rate_hz: float, seed: int = 4) -> list[Request]:
    """Attach seeded Poisson arrival times (mean rate rate_hz) to a serving
    configuration's requests."""
    rng = np.random.default_rng(seed + 1000)
    t = 0.0
    reqs = []
    for i, r in enumerate(cfg["requests"]):
        t += float(rng.exponential(1.0 / rate_hz))
        reqs.append(Request(i, r["grid"], r["flow"], r["seed"], r["steps"], t))
    return reqs
