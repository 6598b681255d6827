"""Benchmark of the fused LES Runge-Kutta path on GB300.

One step = one time step of the whole path: the CFL time-step reduction, five
fused residual/update stages and their boundary fills, on the 256 x 192 x 192
mapped jet grid (9.44e6 points; the paper's scalability workload shape,
arXiv 2003.09926 Section 5.1).  Throughput is reported in Mpt-stage/s =
grid points x 5 stages x steps / time / 1e6.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Headline value: FP32 state and fluxes, metric terms generated in FP64 and
stored in FP32 (P32), inputs resident in HBM, device-timed with CUDA events
on the grid's stream.  Also reported: P32_M64 (FP64-stored metrics; the flux
arithmetic consumes them in FP32, so its results equal P32's) and plain FP64
(P64) variants, the FP32 error against FP64 on the same workload, the fused stage kernel against the
measured HBM roofline, an end-to-end number through the public C ABI with
host buffers, and the CPU FP64 oracle timed on the host cores.

Under torchrun (N > 1) every rank advances its own independent grid (the
batched/served workloads shard by grid with no data exchange): weak scaling,
value = points x stages x steps summed over ranks / max rank time.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpt-stage/s FP32-batched vs plain FP64 at stated err; HBM GB/s; p50/p99 latency"
UNIT = "Mpt-stage/s"
HBM_FALLBACK_GBS = 6800.0
# algorithmic bytes per point-stage of the fused stage kernel: reads of
# Q^(l-1) and Q^(0), write of Q^(l) (5 values each), metric terms S (9) + J;
# stage 1 reads Q^(0) once, so the 5-stage average is (4 x full + 1 x less) / 5
ES = {0: 8, 1: 4, 2: 4}
MS = {0: 8, 1: 8, 2: 4}


# algorithmic flops per point-stage of the fused stage (hand count of the
# method's formulas, each face flux formed once; add, mul = 1, fma = 2,
# div / sqrt / pow = 1 each): conversion 15, node gradients 85, Sutherland 6,
# Smagorinsky 24, stress and heat flux 41, sound speed 1, per-direction node
# fluxes, radii and sensors 180, three face fluxes 168, residual 25, update 11
FLOPS_PER_POINT_STAGE = 556


def bytes_per_point_stage(prec: int) -> float:
    es, ms = ES[prec], MS[prec]
    full = 15 * es + 10 * ms
    first = 10 * es + 10 * ms
    return (4 * full + first) / 5.0


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[4 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows),
                "power_w_max": max((num(r[2]) or 0.0) for r in self.rows)}


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


# stage kernel source files and names per precision (0 P64, 1 P32_M64, 2 P32)
# sources whose change invalidates a recorded DRAM traffic figure: the
# kernel and its headers, and jz_api.cu (TMA tensor maps, default tile shape)
STAGE_SOURCES = {2: ("jz_stage_v.cu", "jz_stage_common.cuh", "jz_fastmath.cuh", "jz_common.cuh", "jz_api.cu"),
                 1: ("jz_stage.cu", "jz_stage_common.cuh", "jz_fastmath.cuh", "jz_common.cuh", "jz_api.cu"),
                 0: ("jz_stage.cu", "jz_stage_common.cuh", "jz_fastmath.cuh", "jz_common.cuh", "jz_api.cu")}
STAGE_KERNELS = {2: "k_stage_v (fused RK stage, vector node records)",
                 1: "k_stage<float,double,32,16> (fused RK stage)",
                 0: "k_stage<double,double,16,16> (fused RK stage)"}


def stage_source_sha(prec: int) -> str:
    h = hashlib.sha256()
    for name in STAGE_SOURCES[prec]:
        with open(os.path.join(ROOT, "paper_2003_09926_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def stage_traffic(prec: int):
    """DRAM bytes per point-stage of the stage kernel from a committed ncu
    capture, if it was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "stage_traffic.json")
    try:
        sha = stage_source_sha(prec)
        with open(p) as fh:
            rec = json.load(fh)
        ent = rec.get(str(prec))
        if ent and ent.get("kernel_sha256") == sha:
            return float(ent["bytes_per_point_stage"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def interior_points(grid: dict) -> int:
    """Nodes the Runge-Kutta stages update (a cylinder's last azimuthal
    plane repeats its first and is not counted)."""
    n = 1
    for a, key in enumerate(("ni", "nj", "nk")):
        per = grid["bc"][2 * a] == 0
        if per:
            n *= grid[key] - 1 if (a == 2 and grid.get("geom", 0) == 1) else grid[key]
        else:
            n *= grid[key] - 2
    return n


def reduce_max(torch, value: float, world: int, device) -> float:
    """Max over ranks (the slowest rank sets the job time)."""
    if world <= 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def weak_value(points_per_rank: int, steps: int, ms: float, world: int) -> float:
    """Whole-job Mpt-stage/s: every rank advances its own grid of
    points_per_rank points by `steps` 5-stage steps within ms (max over ranks)."""
    return world * points_per_rank * 5 * steps / (ms / 1e3) / 1e6


def time_steps(jz, torch, g, steps: int, cfl: float, world: int):
    """Device time of `steps` graph-replayed steps (CUDA events on the grid's
    stream, barrier and synchronize on both sides), max over ranks."""
    dist = torch.distributed
    g.nsteps(1, cfl=cfl)  # the step graph is captured before the timed region
    launches0 = jz.jz_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(g.stream)
    g.nsteps(steps, cfl=cfl)
    ev1.record(g.stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = jz.jz_launch_count() - launches0
    ms = reduce_max(torch, ms, world, "cuda")
    return ms, launches


def profile_steps(jz, torch, g, steps: int, cfl: float):
    """Per-kernel-class device times of `steps` steps launched one by one with
    CUDA events around every launch (outside the timed region):
    ([ms per class], [launches per class])."""
    torch.cuda.synchronize()
    jz.jz_profile_begin(g.h)
    for _ in range(steps):
        g.step(cfl=cfl)
    prof = jz.jz_profile_read(g.h)
    jz.jz_profile_end(g.h)
    return prof


def host_cpu() -> dict:
    """nproc and the CPU model of this host (from /proc/cpuinfo, else lscpu)."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.split(":")[0].strip() in ("Model name", "Vendor ID"):
                    model = line.split(":", 1)[1].strip()
                    if line.startswith("Model name"):
                        break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


# Riemann far-field branch of a boundary value (the boundary-condition
# reading R8): 0 supersonic inflow (u_n <= -c), 1 subsonic with the outside
# entropy, 2 subsonic with the inside entropy, 3 supersonic outflow
# (u_n >= c); the subsonic split is the sign of the characteristic average
# u_n + 2 (c - c_inf) / (gamma - 1) against air at rest (c_inf = 1).  With
# margin=True also returns the distance of the state to the nearest of the
# three switches (|u_n - c|, |u_n + c|, |u_n + 2 (c - 1)/(gamma - 1)|).
def riemann_branch(q, n, gamma=1.4, margin=False):
    rho = q[0]
    u = q[1:4] / rho
    p = (gamma - 1.0) * (q[4] - 0.5 * rho * (u * u).sum(axis=0))
    c = np.sqrt(gamma * p / rho)
    un = (u * n).sum(axis=0)
    split = un + 2.0 * (c - 1.0) / (gamma - 1.0)
    br = np.where(un >= c, 3, np.where(un <= -c, 0, np.where(split > 0.0, 2, 1)))
    if margin:
        return br, np.minimum(np.minimum(np.abs(un - c), np.abs(un + c)), np.abs(split))
    return br


# Stated FP32 bound per node class after the 256x192x192 configuration's
# 200 steps (max |FP32 - FP64| relative to max|v|, worst variable)
FP32_CLASS_BOUNDS = {"interior_d3plus": 5e-5, "interior_d2": 1e-4, "interior_d1": 5e-4, "inflow_face": 1e-6,
                     "farfield_face_clear_of_switch": 5e-4, "farfield_face_near_switch": 0.2}
FP32_BOUNDS_STEPS = 200


# Far-field face nodes closer than this (in velocity units, c_inf = 1) to a
# branch switch in either state are counted as "near a switch": the FP32
# kernel takes the branch decision in its own arithmetic, where 5c - 5 and
# u_n carry errors of a few 1e-6, and the FP32 state at the adjacent node
# differs from the FP64 one by about 1e-5 in these quantities.
BRANCH_MARGIN = 2e-4


def error_classes(Q, Qref, S, bc, gamma=1.4):
    """FP32-vs-FP64 error of every node, by class: inflow-face nodes;
    far-field face nodes whose Riemann branch (riemann_branch, from the
    adjacent interior node and the outward unit normal S^k/|S^k| of the face
    that sets the node: later faces in the order y-, y+, z-, z+, x+, x- win)
    is the same in both states and at least BRANCH_MARGIN from every switch,
    and the others (near a switch, where the two precisions may decide
    differently); nodes at distance 1, 2 and >= 3 from the nearest
    non-periodic face.  Q, Qref: [5][nk][nj][ni];
    S: [>= 9][nk][nj][ni] metrics; bc: the six face kinds (0 periodic, 1
    inflow, 2 far field).  Error of a class: max over variables of
    max|Q - Qref| over its nodes / max|Qref| over all nodes."""
    nk, nj, ni = Q.shape[1:]
    n = (ni, nj, nk)
    big = 1 << 30
    idx = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")  # k, j, i
    dist = np.full((nk, nj, ni), big)
    for d in range(3):
        if bc[2 * d] != 0:
            a = idx[2 - d]
            dist = np.minimum(dist, np.minimum(a, n[d] - 1 - a))
    face = np.full((nk, nj, ni), -1)
    for f in (2, 3, 4, 5, 1, 0):
        d = f // 2
        if bc[f] == 0:
            continue
        a = idx[2 - d]
        face[a == (0 if f % 2 == 0 else n[d] - 1)] = f
    scale = np.abs(Qref).reshape(5, -1).max(axis=1)
    scale = np.where(scale > 0, scale, 1.0)  # an all-zero variable: absolute error
    diff = np.abs(Q - Qref)

    def stat(mask):
        cnt = int(mask.sum())
        if cnt == 0:
            return {"nodes": 0, "max_rel": 0.0, "max_rel_per_variable": [0.0] * 5}
        per = [float(diff[v][mask].max() / scale[v]) for v in range(5)]
        return {"nodes": cnt, "max_rel": max(per), "max_rel_per_variable": per}

    out = {}
    inflow = np.isin(face, [f for f in range(6) if bc[f] == 1])
    out["inflow_face"] = stat(inflow)
    ff = np.zeros_like(inflow)
    differs = np.zeros_like(inflow)
    for f in range(6):
        if bc[f] != 2:
            continue
        m = face == f
        if not m.any():
            continue
        kk, jj, ii = np.nonzero(m)
        ci = [np.clip(ii, 1, ni - 2), np.clip(jj, 1, nj - 2), np.clip(kk, 1, nk - 2)]
        d = f // 2
        sg = -1.0 if f % 2 == 0 else 1.0
        nv = np.stack([S[3 * d + e][kk, jj, ii] for e in range(3)])
        nv = sg * nv / np.sqrt((nv * nv).sum(axis=0))
        b32, m32 = riemann_branch(Q[:, ci[2], ci[1], ci[0]], nv, gamma, margin=True)
        b64, m64 = riemann_branch(Qref[:, ci[2], ci[1], ci[0]], nv, gamma, margin=True)
        ff[kk, jj, ii] = True
        differs[kk, jj, ii] = (b32 != b64) | (np.minimum(m32, m64) < BRANCH_MARGIN)
    out["farfield_face_clear_of_switch"] = stat(ff & ~differs)
    out["farfield_face_near_switch"] = stat(ff & differs)
    out["interior_d1"] = stat(dist == 1)
    out["interior_d2"] = stat(dist == 2)
    out["interior_d3plus"] = stat(dist >= 3)
    out["all_nodes"] = stat(np.ones_like(inflow))
    return out


def cpu_oracle_baseline(cfg: dict, sample_shape=(256, 192, 192)):
    """The oracle as it stands on the host cores: one RK step of the same jet
    workload, timed (metric generation excluded)."""
    import oracle
    from paper_2003_09926_gb300 import workloads as W
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    grid = W.jet_grid(*sample_shape, map_amp=cfg["grid"]["map_amp"], map_seed=cfg["grid"]["map_seed"])
    o = oracle.Oracle(grid, cfg["flow"])
    Q = o.init(cfg["seed"])
    t0 = time.perf_counter()
    o.step(Q, cfl=cfg["cfl"])
    sec = time.perf_counter() - t0
    pts = interior_points(grid)
    # the same per-point arithmetic on one core: 3 steps of the 48x32x32 jet
    c0 = W.config0()
    oracle.set_threads(1)
    o1 = oracle.Oracle(c0["grid"], c0["flow"])
    Q1 = o1.init(c0["seed"])
    t1 = time.perf_counter()
    o1.run(Q1, 3, cfl=c0["cfl"])
    sec1 = time.perf_counter() - t1
    # the 1e9-point configuration's jet and mapping on a 256^3 sub-grid, one
    # RK step on all cores, per point-stage
    oracle.set_threads(cores)
    c2 = W.config2()
    g2 = W.jet_grid(256, 256, 256, map_amp=c2["grid"]["map_amp"], map_seed=c2["grid"]["map_seed"])
    o2 = oracle.Oracle(g2, c2["flow"])
    Q2 = o2.init(c2["seed"])
    t2 = time.perf_counter()
    o2.step(Q2, cfl=c2["cfl"])
    sec2 = time.perf_counter() - t2
    del o2, Q2
    return {"value": pts * 5 / sec / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle", **host_cpu(),
            "sample": f"one RK step (5 stages) of the {sample_shape[0]}x{sample_shape[1]}x{sample_shape[2]} mapped jet "
                      f"grid in FP64, OpenMP over k-planes, {sec:.1f} s",
            "single_thread": {"value": interior_points(c0["grid"]) * 5 * 3 / sec1 / 1e6, "unit": UNIT, "cores": 1,
                              "sample": f"3 RK steps of the 48x32x32 jet in FP64 on one core, {sec1:.2f} s"},
            "c2_subgrid": {"value": interior_points(g2) * 5 / sec2 / 1e6, "unit": UNIT, "cores": cores,
                           "sample": f"one RK step of a 256x256x256 sub-grid of the 1024x1024x960 jet and mapping "
                                     f"in FP64, OpenMP over k-planes, {sec2:.1f} s"}}


def bench_batched(jz, torch, W, local: int, steps: int, steps64: int, cfl: float = 0.5):
    """64 uneven jet grids (32^3 .. 160x128x128), FP32, one persistent launch
    per stage for all grids (graph-replayed), against plain FP64 one grid at a
    time.  The tile shape and k-chunk length are chosen by the autotuner."""
    from paper_2003_09926_gb300 import autotune
    cfg = W.config3()
    cases = [(c["grid"], c["flow"]) for c in cfg["cases"]]
    choice = autotune.tune_batch(cases, cfl=cfl, device=local)
    stream = torch.cuda.Stream(device=local)
    grids = [jz.Grid(c["grid"], stream=stream, device=local).init(c["flow"], c["seed"]) for c in cfg["cases"]]
    for g in grids:
        autotune.apply(g, choice)
    pts = sum(interior_points(c["grid"]) for c in cfg["cases"])
    b = jz.Batch(grids, stream=stream)
    b.nsteps(3, cfl)  # warm-up and graph capture
    stream.synchronize()
    l0 = jz.jz_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.nsteps(steps, cfl)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    launches = jz.jz_launch_count() - l0
    b.close()
    for g in grids:
        g.close()
    # plain FP64, one grid at a time (graph-replayed single-grid steps)
    s64 = torch.cuda.Stream(device=local)
    g64 = [jz.Grid(dict(c["grid"], precision=W.P64), stream=s64, device=local).init(c["flow"], c["seed"])
           for c in cfg["cases"]]
    for g in g64:
        g.nsteps(1, cfl=cfl)
    s64.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(s64)
    for g in g64:
        g.nsteps(steps64, cfl=cfl)
    f1.record(s64)
    f1.synchronize()
    ms64 = f0.elapsed_time(f1)
    for g in g64:
        g.close()
    v32 = pts * 5 * steps / (ms / 1e3) / 1e6
    v64 = pts * 5 * steps64 / (ms64 / 1e3) / 1e6
    return {"workload": "c3: 64 jet grids 32^3..160x128x128 (seed 3), M~U[1.2,2], Re~U[5e5,2e6]",
            "points_updated": pts, "fp32_batched": {"value": v32, "unit": UNIT, "steps": steps, "ms": ms,
                                                    "kernel_launches": launches, "kc": choice["kc"],
                                                    "tile": list(choice["shape"]) if choice["shape"] else None,
                                                    "launches_per_step": launches / steps},
            "fp64_one_grid_at_a_time": {"value": v64, "unit": UNIT, "steps": steps64, "ms": ms64},
            "speedup": v32 / v64}


def bench_cylinder(jz, torch, W, local: int, steps: int, steps64: int, cfl: float = 0.5):
    """The paper's own geometry at its mesh 6 (Tab. mesh: 256 x 128 x 361,
    about 11.8 M points): the cylindrical jet grid with the centreline
    treatment, FP32 (vector-record kernel) and plain FP64, graph-replayed
    steps timed with CUDA events."""
    out = {"workload": "paper mesh 6: cylinder 256x128x361 (axial x radial x azimuthal), jet, CFL 0.5"}
    for prec, n in ((W.P32, steps), (W.P64, steps64)):
        grid = W.cyl_grid(256, 128, 361, precision=prec)
        stream = torch.cuda.Stream(device=local)
        g = jz.Grid(grid, stream=stream, device=local).init(W.jet_flow(), 1)
        ms, launches = time_steps(jz, torch, g, n, cfl, 1)
        pts = interior_points(grid)
        d = g.diagnostics()
        out[W.PRECISION_NAMES[prec]] = {"value": pts * 5 * n / (ms / 1e3) / 1e6, "unit": UNIT, "steps": n,
                                        "ms_per_step": ms / n, "points_updated": pts,
                                        "launches_per_step": launches / n, "finite": d["nonfinite"] == 0}
        g.close()
    return out


def bench_mesh_table(jz, torch, W, local: int, steps: int = 3, cfl: float = 0.5):
    """The paper's thirteen scalability meshes (Tab. mesh: 32 x 32 x 361 ..
    1700 x 1700 x 361, 3.7e5 .. 1.0e9 points) as cylindrical jet grids in
    FP32 on one GPU: per mesh, graph-replayed steps timed with CUDA events
    (at least `steps`, more on the small meshes so that every mesh is timed
    over about 5e7 point-steps, at most 50 steps), the throughput and its
    fraction of the HBM roofline at the algorithmic 96 B per point-stage."""
    peak, peak_kind = measured_hbm_peak()
    rows = []
    for ni, nj in W.PAPER_MESHES:
        grid = W.cyl_grid(ni, nj, 361, precision=W.P32)
        stream = torch.cuda.Stream(device=local)
        g = jz.Grid(grid, stream=stream, device=local).init(W.jet_flow(), 1)
        n = max(steps, min(50, round(5e7 / (ni * nj * 361))))
        ms, _ = time_steps(jz, torch, g, n, cfl, 1)
        pts = interior_points(grid)
        v = pts * 5 * n / (ms / 1e3) / 1e6
        rows.append({"mesh": [ni, nj, 361], "points": ni * nj * 361, "points_updated": pts, "steps": n,
                     "ms_per_step": ms / n,
                     "value": v, "hbm_frac": v * 1e6 * 96.0 / (peak * 1e9) if peak else None,
                     "finite": g.diagnostics()["nonfinite"] == 0})
        g.close()
        del g
        torch.cuda.empty_cache()
    return {"workload": "paper Tab. mesh 1-13 as cylinders (xi x eta x 361), jet, P32", "unit": UNIT,
            "min_steps": steps, "hbm_peak_gbs": peak, "peak_kind": peak_kind, "meshes": rows}


def bench_billion(jz, torch, W, local: int, steps: int, cfl: float = 0.5):
    """The paper's largest mesh size (Tab. mesh: about 1e9 points) on one GPU:
    c2, 1024 x 1024 x 960 mapped jet in FP32 (state, fluxes and stored
    metrics; about 104 GB of HBM), graph-replayed steps."""
    cfg = W.config2()
    grid = cfg["grid"]
    stream = torch.cuda.Stream(device=local)
    g = jz.Grid(grid, stream=stream, device=local).init(cfg["flow"], cfg["seed"])
    ms, launches = time_steps(jz, torch, g, steps, cfl, 1)
    pts = interior_points(grid)
    d = g.diagnostics()
    out = {"workload": "c2: 1024x1024x960 mapped jet (1.007e9 points), P32", "value": pts * 5 * steps / (ms / 1e3) / 1e6,
           "unit": UNIT, "steps": steps, "ms_per_step": ms / steps, "points_updated": pts,
           "device_bytes": g.nbytes, "launches_per_step": launches / steps, "finite": d["nonfinite"] == 0}
    g.close()
    del g
    torch.cuda.empty_cache()
    return out


def fifo_extrapolation(trace, rate_mpt: float) -> dict:
    """Latencies of serving `trace` one case at a time in arrival order at a
    fixed rate (Mpt-stage/s): start = max(arrival, previous finish),
    finish = start + case work / rate."""
    from paper_2003_09926_gb300 import serve
    t, lat, work = 0.0, [], 0.0
    for r in sorted(trace, key=lambda r: (r.arrival, r.rid)):
        w = serve.updated_points(r.grid) * 5 * r.steps
        t = max(t, r.arrival) + w / (rate_mpt * 1e6)
        lat.append(t - r.arrival)
        work += w
    span = t - min(r.arrival for r in trace)
    return {"completed": len(lat), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(np.mean(lat)),
            "makespan_s": span, "throughput_mpt_stage_s": work / span / 1e6}


def bench_serving(jz, torch, W, local: int, capacity: float, nreq: int = 256, base64_n: int = 4,
                  pts_hi: float = 2e7, orders=(), fill: int = 4 * 10**6):
    """Continuous serving of the trace: log-uniform 1e5..pts_hi points per
    case (the configuration's 2e7 by default), 50..500 steps, Poisson
    arrivals at 70% of the measured batched capacity, 150 GB HBM budget.
    Headline: prioritised streams (at most 2 resident cases, the oldest on
    the highest-priority stream, 20-step chunks, a case joining the oldest
    only while its work is at most a quarter of the oldest's remaining work); optionally the time-slice
    server with batched launches in the given slice orders; against the
    same trace served one case at a time in FP32, and in plain FP64 on its
    first cases with the full trace extrapolated at the FP64 rate measured
    there."""
    from paper_2003_09926_gb300 import serve
    cfg = W.config4(nreq=nreq, pts_hi=pts_hi)
    work = np.mean([interior_points(r["grid"]) * 5 * r["steps"] for r in cfg["requests"]])
    rate = 0.7 * capacity * 1e6 / work
    trace = serve.poisson_trace(cfg, rate)
    out = {"workload": f"c4 trace: {nreq} cases, log-uniform 1e5..{pts_hi:.0e} points, 50..500 steps, seed 4",
           "arrival_rate_hz": rate, "budget_bytes": 150 * 10**9}
    srv = serve.PriorityServer(150 * 10**9, max_running=2, chunk_steps=20, device=local, fill_ratio=0.25)
    out["fp32_continuous_priority_streams"] = dict(
        serve.summarize(srv.run(trace)), max_running=2, chunk_steps=20, fill_ratio=0.25, chunks=srv.chunks,
        peak_resident_bytes=srv.peak_bytes,
        policy="cases admitted in arrival order as memory and one of 2 slots free up, a case beside the oldest "
               "only while its work is at most 0.25 of the oldest's remaining work; each advances with its own "
               "graph-replayed steps, 20 at a time, on the stream of its arrival rank (oldest = highest priority), "
               "so later cases run in the capacity the oldest leaves idle")
    for order in orders:
        srv = serve.Server(150 * 10**9, slice_steps=10, device=local, fill_points=fill, order=order)
        res = srv.run(trace)
        out[f"fp32_time_slices_{order}"] = dict(serve.summarize(res), fill_points=fill, order=order, slice_steps=10,
                                                peak_resident_bytes=srv.peak_bytes, slices=srv.slices)
    out["fp32_one_at_a_time"] = serve.summarize(serve.serve_one_at_a_time(trace, W.P32, device=local))
    first = serve.serve_one_at_a_time(trace[:base64_n], W.P64, device=local)
    busy = sum(r.finished - r.admitted for r in first)
    w64 = sum(r.points * 5 * r.steps for r in first)
    rate64 = w64 / busy / 1e6
    out["fp64_one_at_a_time_first_cases"] = dict(serve.summarize(first), cases=base64_n)
    out["fp64_one_at_a_time_extrapolated"] = dict(
        fifo_extrapolation(trace, rate64), fp64_rate_mpt_stage_s=rate64,
        note=f"extrapolated, not measured: every case of the trace served in arrival order at the FP64 rate "
             f"measured on the first {base64_n} cases ({rate64:.0f} Mpt-stage/s)")
    return out


def run_reference(args, rank, world):
    """Reference arm: the CPU FP64 oracle on the host cores, same metric."""
    if rank != 0:
        return 0
    from paper_2003_09926_gb300 import workloads as W
    import oracle
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    cfg = W.config1()
    shape = (64, 48, 48)  # bounded sample of the 256x192x192 workload per step
    grid = W.jet_grid(*shape, map_amp=cfg["grid"]["map_amp"], map_seed=cfg["grid"]["map_seed"])
    o = oracle.Oracle(grid, cfg["flow"])
    Q = o.init(cfg["seed"])
    for _ in range(args.warmup):
        o.step(Q, cfl=cfg["cfl"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(Q, cfl=cfg["cfl"])
    sec = time.perf_counter() - t0
    pts = interior_points(grid)
    value = pts * 5 * args.steps / sec / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "c1_jet_256x192x192 (per step: 64x48x48 sample of the same jet and mapping)",
                       "precision": "FP64 oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", **host_cpu(),
                             "sample": f"{args.steps} RK steps of a 64x48x48 sample of the mapped jet workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=0, help="timed steps of the FP64 variant (default steps/10)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-grid batched measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-cylinder", action="store_true", help="skip the cylindrical-grid measurement")
    ap.add_argument("--no-billion", action="store_true", help="skip the 1e9-point measurement")
    ap.add_argument("--no-mesh-table", action="store_true",
                    help="skip the paper's thirteen scalability meshes as cylinders (3.7e5 .. 1e9 points, about 10 s)")
    ap.add_argument("--err-steps", type=int, default=200,
                    help="steps of the FP32-vs-FP64 error runs (the 256x192x192 configuration's 200)")
    ap.add_argument("--serving-quick", action="store_true",
                    help="serve a bounded 32-case trace of at most 2e6 points instead of the configuration's 256 "
                         "cases of 1e5..2e7 points (several minutes)")
    ap.add_argument("--serving-orders", default="",
                    help="also serve the trace with the time-slice server in these comma-separated slice orders "
                         "(remaining, arrival, head)")
    args = ap.parse_args(argv)
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    import torch
    from paper_2003_09926_gb300 import build as B
    from paper_2003_09926_gb300 import jz
    from paper_2003_09926_gb300 import workloads as W

    B.build()
    jz.lib()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))

    head = W.P32
    cfg = W.config1(precision=head)
    grid = cfg["grid"]
    pts = interior_points(grid)
    results = {}
    clocks = None
    prof = prof64 = None
    launches = 0
    for prec in (head, W.P32_M64, W.P32_S64, W.P64):
        g = jz.Grid(dict(grid, precision=prec), device=local).init(cfg["flow"], cfg["seed"] + rank)
        steps = args.steps if prec != W.P64 else (args.fp64_steps or max(3, args.steps // 10))
        for _ in range(args.warmup):
            g.step(cfl=cfg["cfl"])
        torch.cuda.synchronize()
        if prec == head:
            with ClockSampler(local) as cs:
                ms, launches = time_steps(jz, torch, g, steps, cfg["cfl"], world)
            clocks = cs.summary()
            prof = profile_steps(jz, torch, g, 20, cfg["cfl"])
        else:
            ms, _ = time_steps(jz, torch, g, steps, cfg["cfl"], world)
            if prec == W.P64:
                prof64 = profile_steps(jz, torch, g, 2, cfg["cfl"])
        results[prec] = {"ms_per_step": ms / steps, "steps": steps, "value": weak_value(pts, steps, ms, world)}
        g.close()
        del g
        torch.cuda.empty_cache()

    # FP32 error against FP64 on this workload after 20 steps from the same state
    err_steps = args.err_steps
    ref = jz.Grid(dict(grid, precision=W.P64), device=local).init(cfg["flow"], cfg["seed"])
    ref.nsteps(err_steps, cfl=cfg["cfl"])
    Qref = ref.download()
    Sref = ref.metrics()
    ref.close()
    del ref
    errors = {}
    for prec in (W.P32_M64, W.P32, W.P32_S64):
        g = jz.Grid(dict(grid, precision=prec), device=local).init(cfg["flow"], cfg["seed"])
        g.nsteps(err_steps, cfl=cfg["cfl"])
        Q = g.download()
        g.close()
        inner = (slice(3, -3),) * 3
        per_var = [float(np.abs(Q[v][inner] - Qref[v][inner]).max() / np.abs(Qref[v]).max()) for v in range(5)]
        errors[W.PRECISION_NAMES[prec]] = {
            "max_rel_interior": max(per_var),
            "max_rel_interior_per_variable": per_var,
            "max_rel_all_nodes": max(float(np.abs(Q[v] - Qref[v]).max() / np.abs(Qref[v]).max()) for v in range(5)),
            "l2_rel": max(float(np.sqrt(np.mean((Q[v] - Qref[v]) ** 2) / np.mean(Qref[v] ** 2))) for v in range(5)),
            "classes": error_classes(Q, Qref, Sref, grid["bc"])}
        # the bounds are stated for the configuration's run length: after a
        # few steps the transverse momenta are still near zero, and errors
        # relative to their maxima read larger
        errors[W.PRECISION_NAMES[prec]]["within_stated_bounds"] = all(
            errors[W.PRECISION_NAMES[prec]]["classes"][k]["max_rel"] <= b
            for k, b in FP32_CLASS_BOUNDS.items()) if err_steps == FP32_BOUNDS_STEPS else None
        del g
    del Qref, Sref

    # end to end through the public C ABI with host buffers: the initial state
    # uploaded from pinned host memory; every step's metric -- the
    # diagnostics (conservation sums, extrema, non-finite count) of the state
    # the step starts from, formed by the step's own time-step reduction --
    # copied to pinned host memory and read on the host one step behind (the
    # host enqueues step s+1 before it waits for step s's record); the final
    # state's diagnostics by one diagnostics pass; the final state downloaded
    g = jz.Grid(dict(grid, precision=head), device=local).init(cfg["flow"], cfg["seed"] + rank)
    g.set_step_diagnostics(True)
    host_in = torch.empty(g.shape, dtype=torch.float64, pin_memory=True).numpy()
    host_out = torch.empty(g.shape, dtype=torch.float64, pin_memory=True).numpy()
    slots = [jz.PinnedDiag(), jz.PinnedDiag()]
    evs = [torch.cuda.Event(), torch.cuda.Event()]

    def run(n):
        seen = []
        for s in range(n):
            g.nsteps(1, cfl=cfg["cfl"])
            g.step_diagnostics_async(slots[s % 2])
            evs[s % 2].record(g.stream)
            if s >= 1:
                evs[(s - 1) % 2].synchronize()
                seen.append(slots[(s - 1) % 2].read())
        evs[(n - 1) % 2].synchronize()
        seen.append(slots[(n - 1) % 2].read())
        g.diagnostics_async(slots[0])  # the state after the last step
        evs[0].record(g.stream)
        evs[0].synchronize()
        seen.append(slots[0].read())
        return seen

    g.download(host_in)
    g.download(host_out)  # both pinned host buffers written once before the timed region
    run(args.warmup)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.upload(host_in)  # synchronous, like the download
    t1 = time.perf_counter()
    seen = run(args.steps)
    t2 = time.perf_counter()
    g.download(host_out)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    e2e_s = t3 - t0
    assert len(seen) == args.steps + 1 and all(d["nonfinite"] == 0 for d in seen)
    assert [d["step"] for d in seen] == list(range(seen[0]["step"], seen[0]["step"] + args.steps + 1))
    e2e_s = reduce_max(torch, e2e_s, world, "cuda")
    state_bytes = host_in.nbytes
    diag_bytes = ctypes.sizeof(jz.Diag) * len(seen)  # the records copied
    e2e = {"value": weak_value(pts, args.steps, 1e3 * e2e_s, world), "unit": UNIT,
           "h2d_bytes_per_step": state_bytes / args.steps,
           "d2h_bytes_per_step": (diag_bytes + state_bytes) / args.steps,
           "split_ms": {"upload": 1e3 * (t1 - t0), "steps": 1e3 * (t2 - t1), "download": 1e3 * (t3 - t2)},
           "note": "initial state uploaded from pinned host memory; every step's diagnostics (of the state the "
                   "step starts from, formed by its time-step reduction) copied to pinned host memory and read "
                   "one step behind; the final state's diagnostics by one pass; final state downloaded"}
    g.close()

    # roofline of the fused stage kernel (dominant kernel) in the headline run
    peak, peak_kind = measured_hbm_peak()
    ms_k, n_k = prof[0][0], prof[1][0]
    stage_ms = ms_k / max(1, n_k)
    bpps = bytes_per_point_stage(head)
    achieved = bpps * pts / (stage_ms / 1e3) / 1e9
    tr = stage_traffic(head)
    total_ms = sum(prof[0])
    stream = torch.cuda.current_stream().cuda_stream
    fp32_peak = jz.jz_fma_peak(False, stream)
    fp64_peak = jz.jz_fma_peak(True, stream)
    fp32_tf = FLOPS_PER_POINT_STAGE * pts / (stage_ms / 1e3) / 1e12
    stage64_ms = prof64[0][0] / max(1, prof64[1][0])
    fp64_tf = FLOPS_PER_POINT_STAGE * pts / (stage64_ms / 1e3) / 1e12
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (tr * pts) if tr else None, "peak_kind": peak_kind,
                "kernel": STAGE_KERNELS[head], "algorithmic_bytes_per_point_stage": bpps,
                "points_per_launch": pts, "avg_launch_ms": stage_ms,
                "share_of_step": ms_k / total_ms if total_ms else None,
                "other_kernels_ms": {"boundary_fill": prof[0][1], "timestep": prof[0][2]},
                "profiled_steps": 20,
                "fp32_alu": {"flops_per_point_stage": FLOPS_PER_POINT_STAGE, "achieved_tflops": fp32_tf,
                             "peak_tflops": fp32_peak, "frac": fp32_tf / fp32_peak if fp32_peak else None,
                             "peak_kind": "measured FP32 FMA chains (jz_fma_peak)"}}
    fp64_roofline = {"bound": "alu", "kernel": STAGE_KERNELS[W.P64], "achieved": fp64_tf, "peak": fp64_peak,
                     "unit": "TFLOP/s", "frac": fp64_tf / fp64_peak if fp64_peak else None,
                     "flops_per_point_stage": FLOPS_PER_POINT_STAGE, "avg_launch_ms": stage64_ms,
                     "peak_kind": "measured FP64 FMA chains (jz_fma_peak)"}

    line = {"metric": METRIC, "value": results[head]["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": results[head]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c1_jet_256x192x192 mapped jet, FP32 state/flux, FP64-generated FP32 metrics (P32)",
                       "grid": [grid["ni"], grid["nj"], grid["nk"]], "points_updated": pts,
                       "precision": "P32", "parallelism": f"{world} independent grid(s), one per GPU",
                       "l2": "inputs larger than L2 (state + metrics 1.0 GB per grid)"},
            "roofline": roofline, "fp64_roofline": fp64_roofline, "gpu_launches": launches, "clocks": clocks,
            "e2e": e2e,
            "variants": {W.PRECISION_NAMES[p]: r for p, r in results.items()},
            "fp32_error_vs_fp64": {"steps": err_steps, "per_mode": errors,
                                   "interior": "nodes at least 3 from every face",
                                   "stated_bounds": FP32_CLASS_BOUNDS, "bounds_steps": FP32_BOUNDS_STEPS,
                                   "classes": "every node by class: inflow face; far-field face nodes whose Riemann branch (supersonic in / subsonic outside entropy / subsonic inside entropy / supersonic out, from the adjacent interior node) is the same in both precisions and at least 2e-4 from every switch, and the others (near a switch: the two precisions may decide differently); nodes at distance 1, 2 and >= 3 from the nearest face"},
            "fp64_vs_fp32_speedup": results[head]["value"] / results[W.P64]["value"]}
    if not args.no_batched:
        line["batched"] = bench_batched(jz, torch, W, local, steps=max(10, args.steps // 5), steps64=2)
    if not args.no_serving:
        cap = line["batched"]["fp32_batched"]["value"] if "batched" in line else results[head]["value"]
        orders = tuple(o for o in args.serving_orders.split(",") if o)
        line["serving"] = (bench_serving(jz, torch, W, local, cap, nreq=32, pts_hi=2e6, orders=orders)
                           if args.serving_quick else bench_serving(jz, torch, W, local, cap, orders=orders))
    if not args.no_cylinder:
        line["cylinder"] = bench_cylinder(jz, torch, W, local, steps=max(10, args.steps // 4), steps64=2)
    if not args.no_billion and world == 1:
        line["billion"] = bench_billion(jz, torch, W, local, steps=max(3, args.steps // 40))
    if not args.no_mesh_table and world == 1:
        line["mesh_table"] = bench_mesh_table(jz, torch, W, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_baseline(cfg)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
