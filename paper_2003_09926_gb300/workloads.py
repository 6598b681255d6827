"""Synthetic workloads: grid descriptors and flow parameters.

Plain parameter sets and seeded generators only -- no arithmetic of the
method lives here.  The jet case follows the scalability and validation set-up
of arXiv 2003.09926 (Section 5.1 and Section 6: perfectly expanded isothermal
Mach 1.4 jet, Re_D = 1.57e6, gamma = 1.4, Pr = 0.72); the grid sizes follow the
paper's mesh table (Section 5.1, Tab. mesh: 3.7e5 .. 1e9 points, ratio-2 growth)
on a Cartesian box x in [0, 30], y, z in [-8, 8] (jet diameter D = 1).
"""
from __future__ import annotations

import math

import numpy as np

BC_PERIODIC, BC_INFLOW, BC_FARFIELD, BC_AXIS = 0, 1, 2, 4
GEOM_BOX, GEOM_CYLINDER = 0, 1
P64, P32_M64, P32, P32_S64 = 0, 1, 2, 3
IC_JET, IC_QUIESCENT = 0, 1
SGS_SMAGORINSKY, SGS_VREMAN = 0, 1
PRECISION_NAMES = {P64: "P64", P32_M64: "P32_M64", P32: "P32", P32_S64: "P32_S64"}

JET_BC = [BC_INFLOW, BC_FARFIELD, BC_FARFIELD, BC_FARFIELD, BC_FARFIELD, BC_FARFIELD]
ALL_PERIODIC = [BC_PERIODIC] * 6


def jet_flow(**over) -> dict:
    """Flow parameters of the jet case (readings of the paper's silent
    constants: Sutherland S1 = 110.4 K / 288.15 K, Smagorinsky C_s = 0.18,
    Pr_t = 0.9, Turkel-Vatsa k2 = 1/4, k4 = 1/256, sigma = 1/2)."""
    f = dict(mach=1.4, re=1.57e6, gamma=1.4, pr=0.72, prt=0.9, cs=0.18, k2=0.25, k4=1.0 / 256.0, sigma=0.5,
             s1=110.4 / 288.15, r0=0.5, theta=0.05, noise=0.01, ic=IC_JET, sgs=SGS_SMAGORINSKY)
    f.update(over)
    return f


def jet_grid(ni: int, nj: int, nk: int, map_amp: float = 0.0, map_seed: int = 0, precision: int = P64) -> dict:
    """Box x in [0,30], y,z in [-8,8], tanh clustering of y and z at |y| = 0.5."""
    return dict(ni=ni, nj=nj, nk=nk, bc=list(JET_BC), lo=[0.0, -8.0, -8.0], hi=[30.0, 8.0, 8.0],
                cluster_r=0.5, stretch_c=0.4, stretch_w=0.5, map_amp=map_amp, map_seed=map_seed,
                precision=precision)


CYL_BC = [BC_INFLOW, BC_FARFIELD, BC_AXIS, BC_FARFIELD, BC_PERIODIC, BC_PERIODIC]


def cyl_grid(ni: int, nj: int, nk: int = 361, length: float = 30.0, radius: float = 8.0, stretch_c: float = 0.4,
             precision: int = P64) -> dict:
    """The paper's cylindrical jet grid (Section 3, Tab. mesh): xi axial on
    [0, length], eta radial on [0, radius] from the centreline with the tanh
    clustering at r = 0.5, zeta azimuthal with nk points (361 in the paper),
    the first and last coinciding."""
    return dict(ni=ni, nj=nj, nk=nk, bc=list(CYL_BC), lo=[0.0, 0.0, 0.0], hi=[length, radius, 2.0 * math.pi],
                cluster_r=0.5, stretch_c=stretch_c, stretch_w=0.5, map_amp=0.0, map_seed=0, precision=precision,
                geom=GEOM_CYLINDER)


# the paper's scalability meshes (Tab. mesh): points in xi (axial) and eta
# (radial), all with 361 azimuthal points
PAPER_MESHES = [(32, 32), (64, 32), (64, 64), (128, 64), (128, 128), (256, 128), (256, 256), (512, 256),
                (512, 512), (1024, 512), (1024, 1024), (2048, 1024), (1700, 1700)]


def periodic_grid(ni: int, nj: int, nk: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), map_amp: float = 0.0,
                  map_seed: int = 0, precision: int = P64) -> dict:
    return dict(ni=ni, nj=nj, nk=nk, bc=list(ALL_PERIODIC), lo=list(lo), hi=list(hi), cluster_r=0.5,
                stretch_c=0.0, stretch_w=0.5, map_amp=map_amp, map_seed=map_seed, precision=precision)


# --- the configurations the measurements use --------------------------------

def config0():
    """Plain FP64 method, 48x32x32 (49,152 points), 20 steps at CFL 0.5."""
    return dict(name="c0_jet_48x32x32", grid=jet_grid(48, 32, 32), flow=jet_flow(), seed=0, steps=20, cfl=0.5)


def config1(precision: int = P64):
    """256x192x192 (9.44e6 points), 2% sinusoidal mapping, 200 steps."""
    return dict(name="c1_jet_256x192x192", grid=jet_grid(256, 192, 192, map_amp=0.02, map_seed=1,
                                                         precision=precision),
                flow=jet_flow(), seed=1, steps=200, cfl=0.5)


def config2():
    """1024x1024x960 (1.007e9 points), config-1 jet + mapping, FP32, 10 steps."""
    return dict(name="c2_jet_1024x1024x960", grid=jet_grid(1024, 1024, 960, map_amp=0.02, map_seed=1,
                                                           precision=P32),
                flow=jet_flow(), seed=1, steps=10, cfl=0.5)


def config3(ngrids: int = 64, seed: int = 3, precision: int = P32):
    """64 uneven jet grids, Ni in {32..160}, Nj = Nk in {32..128} (step 16),
    Mach ~ U[1.2, 2.0], Re_D ~ U[5e5, 2e6], init seed 3000 + g, 100 steps."""
    rng = np.random.default_rng(seed)
    cases = []
    for gi in range(ngrids):
        ni = int(rng.choice(np.arange(32, 161, 16)))
        nj = int(rng.choice(np.arange(32, 129, 16)))
        mach = float(rng.uniform(1.2, 2.0))
        re = float(rng.uniform(5e5, 2e6))
        cases.append(dict(grid=jet_grid(ni, nj, nj, precision=precision), flow=jet_flow(mach=mach, re=re),
                          seed=3000 + gi))
    return dict(name="c3_batch64", cases=cases, steps=100, cfl=0.5)


def config4(nreq: int = 256, seed: int = 4, precision: int = P32, pts_lo: float = 1e5, pts_hi: float = 2e7):
    """Serving trace: log-uniform points per request in [1e5, 2e7] with shape
    Ni:Nj:Nk ~ 1.5:1:1, steps uniform in {50..500}, parameters as config 3.
    Arrival times are attached by the caller (Poisson at a chosen rate)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(nreq):
        pts = math.exp(rng.uniform(math.log(pts_lo), math.log(pts_hi)))
        nj = max(8, int(round((pts / 1.5) ** (1.0 / 3.0))))
        ni = max(8, int(round(1.5 * nj)))
        steps = int(rng.integers(50, 501))
        mach = float(rng.uniform(1.2, 2.0))
        re = float(rng.uniform(5e5, 2e6))
        reqs.append(dict(grid=jet_grid(ni, nj, nj, precision=precision), flow=jet_flow(mach=mach, re=re),
                         seed=4000 + r, steps=steps))
    return dict(name="c4_serve", requests=reqs, cfl=0.5)
