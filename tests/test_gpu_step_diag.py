"""Diagnostics formed by the steps' own time-step reduction
(jz_set_step_diagnostics): the record of a step is the diagnostics of the
state the step starts from, the same as a separate jz_diagnostics pass over
that state -- extrema, non-finite count, time, step and dt exactly, the five
volume sums up to the rounding of another summation order -- and switching
them on leaves the stepping bitwise unchanged."""
import numpy as np
import pytest

from paper_2003_09926_gb300 import workloads as W

import states as ST

pytestmark = pytest.mark.gpu

# relative agreement of the volume sums: FP64 sums in another order; FP32
# compensated (TwoSum) per-thread sums folded to FP64
SUM_REL = {W.P64: 1e-12, W.P32_M64: 1e-9, W.P32: 1e-9}


@pytest.fixture(scope="module")
def jz():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09926_gb300 import build, jz as J
    build.build()
    J.lib()
    return J


def _record(jz, g):
    out = jz.PinnedDiag()
    g.step_diagnostics_async(out)
    g.synchronize()
    return out.read()


def _same(rec, ref, prec):
    for k in ("time", "step", "dt", "rho_min", "rho_max", "p_min", "p_max", "mach_max", "nonfinite"):
        assert rec[k] == ref[k], (k, rec[k], ref[k])
    s, r = np.asarray(rec["sum"]), np.asarray(ref["sum"])
    assert np.all(np.abs(s - r) <= SUM_REL[prec] * np.abs(r).max()), (s, r)


@pytest.mark.parametrize("prec", [W.P64, W.P32_M64, W.P32])
def test_step_record_is_the_diagnostics_of_the_step_state(jz, prec):
    grid = W.jet_grid(45, 27, 22, map_amp=0.03, map_seed=2, precision=prec)
    g = jz.Grid(grid).init(W.jet_flow(), 4)
    g.nsteps(3, cfl=0.5)
    ref = g.diagnostics()
    g.set_step_diagnostics(True)
    g.nsteps(1, cfl=0.5)
    _same(_record(jz, g), ref, prec)
    g.close()


@pytest.mark.parametrize("prec", [W.P64, W.P32])
def test_step_diagnostics_leave_the_stepping_unchanged(jz, prec):
    grid = W.jet_grid(40, 24, 20, map_amp=0.03, map_seed=3, precision=prec)
    a = jz.Grid(grid).init(W.jet_flow(), 5)
    b = jz.Grid(grid).init(W.jet_flow(), 5)
    b.set_step_diagnostics(True)
    a.nsteps(6, cfl=0.5)
    b.nsteps(6, cfl=0.5)
    # after graph-replayed steps the record is that of the state the last
    # step started from (step 5); read before jz_diagnostics replaces it
    rec = _record(jz, b)
    c = jz.Grid(grid).init(W.jet_flow(), 5)
    c.nsteps(5, cfl=0.5)
    _same(rec, c.diagnostics(), prec)
    np.testing.assert_array_equal(a.download(), b.download())
    da, db = a.diagnostics(), b.diagnostics()
    assert da["time"] == db["time"] and da["dt"] == db["dt"] and da["step"] == db["step"] == 6
    for g in (a, b, c):
        g.close()


def test_fixed_dt_steps_form_the_record_by_the_diagnostics_pass(jz):
    grid = W.periodic_grid(30, 18, 12, hi=(2.0, 1.5, 1.2), map_amp=0.2, map_seed=5, precision=W.P32)
    g = jz.Grid(grid).init(W.jet_flow(re=1e3), 0)
    g.upload(ST.random_state((12, 18, 30), seed=2))
    ref = g.diagnostics()
    g.set_step_diagnostics(True)
    g.nsteps(1, dt=1e-3)
    rec = _record(jz, g)
    for k in rec:
        assert np.all(np.asarray(rec[k]) == np.asarray(ref[k])), k
    g.close()


def test_non_finite_nodes_are_counted_and_left_out(jz):
    grid = W.jet_grid(34, 20, 18, precision=W.P32)
    g = jz.Grid(grid).init(W.jet_flow(), 1)
    Q = g.download()
    Q[0, 5, 7, 9] = np.nan
    Q[3, 2, 2, 2] = np.inf
    g.upload(Q)
    ref = g.diagnostics(allow_nonfinite=True)
    assert ref["nonfinite"] == 2
    g.set_step_diagnostics(True)
    g.nsteps(1, cfl=0.5)
    _same(_record(jz, g), ref, W.P32)
    g.close()
