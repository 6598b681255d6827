"""Batched execution: many uneven grids advanced by one persistent stage
launch per stage (plus one batched time-step and boundary launch), captured
in a CUDA graph.  Each grid keeps its own CFL time step; the per-point
arithmetic does not depend on the batch, so every grid's state must be
bitwise the one it reaches when stepped alone."""
import numpy as np
import pytest

from paper_2003_09926_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(40, 24, 20), (33, 17, 19), (64, 32, 32), (20, 40, 12), (48, 16, 24), (3, 3, 3)]


@pytest.fixture(scope="module")
def jz():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09926_gb300 import build, jz as J
    build.build()
    J.lib()
    return J


@pytest.mark.parametrize("prec", [W.P32, W.P64])
def test_batch_equals_grids_alone(jz, prec):
    import torch
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(8)
    cases = []
    for gi, sh in enumerate(SHAPES):
        flow = W.jet_flow(mach=float(rng.uniform(1.2, 2.0)), re=float(rng.uniform(5e5, 2e6)))
        cases.append((W.jet_grid(*sh, map_amp=0.03 * (gi % 2), map_seed=gi, precision=prec), flow, 100 + gi))
    batch_grids = [jz.Grid(g, stream=stream).init(f, s) for g, f, s in cases]
    jz.jz_set_tiling(batch_grids[2].h, 5)  # uneven chunking inside the batch
    b = jz.Batch(batch_grids, stream=stream)
    b.nsteps(4, cfl=0.5)
    b.nsteps(3, cfl=0.5)
    stream.synchronize()
    for (g, f, s), bg in zip(cases, batch_grids):
        alone = jz.Grid(g).init(f, s)
        alone.nsteps(7, cfl=0.5)
        np.testing.assert_array_equal(bg.download(), alone.download())
        da, db = alone.diagnostics(), bg.diagnostics()
        assert db["step"] == 7 and db["time"] == da["time"] and db["dt"] == da["dt"]
    b.close()


@pytest.mark.parametrize("prec", [W.P32, W.P64, W.P32_M64, W.P32_S64])
def test_mixed_flow_models_equal_their_own_builds(jz, prec):
    """The stage kernels are compiled per flow model with constant flags
    (FP32 vector-record kernel: Smagorinsky, Vreman, inviscid, all with
    sigma = 1/2; the scalar kernels of the other modes: Smagorinsky) and once
    with the flags read at run time.  A batch whose grids differ in model
    runs the runtime build; stepped alone, each grid runs its own build (the
    runtime one for the models without a constant-flag build).  The states
    must agree bitwise: the builds differ in branches, not in the arithmetic
    of a node."""
    import torch
    flows = [W.jet_flow(), W.jet_flow(re=5e3, sgs=W.SGS_VREMAN), W.jet_flow(re=0.0, cs=0.0),
             W.jet_flow(re=4e3, cs=0.0), W.jet_flow(sigma=0.7)]
    shapes = [(36, 22, 18), (33, 17, 19), (40, 24, 20), (20, 18, 12), (24, 20, 14)]
    cases = [(W.jet_grid(*sh, map_amp=0.03, map_seed=k, precision=prec), f, 40 + k)
             for k, (sh, f) in enumerate(zip(shapes, flows))]
    stream = torch.cuda.Stream()
    batch_grids = [jz.Grid(g, stream=stream).init(f, s) for g, f, s in cases]
    b = jz.Batch(batch_grids, stream=stream)
    b.nsteps(4, cfl=0.5)
    stream.synchronize()
    for (g, f, s), bg in zip(cases, batch_grids):
        alone = jz.Grid(g).init(f, s)
        alone.nsteps(4, cfl=0.5)
        np.testing.assert_array_equal(bg.download(), alone.download())
        alone.close()
    b.close()


def test_batch_rejects_mixed_precision(jz):
    import torch
    s = torch.cuda.Stream()
    a = jz.Grid(W.jet_grid(20, 12, 10, precision=W.P32), stream=s).init(W.jet_flow(), 0)
    c = jz.Grid(W.jet_grid(20, 12, 10, precision=W.P64), stream=s).init(W.jet_flow(), 0)
    with pytest.raises(jz.JzError) as ei:
        jz.Batch([a, c], stream=s)
    assert ei.value.code == jz.JZ_EINVAL


def test_autotuner_chooses_shape_and_chunk(jz):
    """The batch autotuner returns one of the built tile shapes and a chunk
    length; applied to the grids, the batched result is bitwise the default
    one (the choice changes the schedule, never the arithmetic)."""
    import torch
    from paper_2003_09926_gb300 import autotune
    cases = [(W.jet_grid(34, 18, 16, precision=W.P32), W.jet_flow()),
             (W.jet_grid(66, 40, 24, precision=W.P32), W.jet_flow(mach=1.6))]
    choice = autotune.tune_batch(cases)
    assert choice["shape"] in autotune.SHAPES and choice["kc"] is not None and choice["ms"] > 0
    stream = torch.cuda.Stream()
    outs = []
    for tuned in (False, True):
        grids = [jz.Grid(d, stream=stream).init(f, 3) for d, f in cases]
        if tuned:
            for g in grids:
                autotune.apply(g, choice)
        b = jz.Batch(grids, stream=stream)
        b.nsteps(3, cfl=0.5)
        stream.synchronize()
        outs.append([g.download() for g in grids])
        b.close()
    for a, c in zip(*outs):
        np.testing.assert_array_equal(a, c)
    one = autotune.tune_grid(cases[0][0], cases[0][1])
    assert one["shape"] in autotune.SHAPES


def _rel_err(got, ref):
    return max(np.abs(got[v] - ref[v]).max() / np.abs(ref[v]).max() for v in range(5))


def test_p64_batch_matches_the_oracle(jz):
    """Direct parity of the batched path: three uneven FP64 jet grids (one
    with the sinusoidal mapping, one chunked in k), each with its own Mach
    and Reynolds numbers and its own CFL time step, advanced five steps in
    one batch, are each within 1e-10 of the CPU oracle run on that grid
    alone (paper Section 4.2, Fig. jazzy: the per-stage sequence)."""
    import torch

    import oracle
    stream = torch.cuda.Stream()
    cases = [(W.jet_grid(40, 24, 20, map_amp=0.03, map_seed=5), W.jet_flow(mach=1.3, re=8e5), 11),
             (W.jet_grid(33, 17, 19), W.jet_flow(mach=1.9, re=1.5e6), 12),
             (W.jet_grid(20, 28, 14, map_amp=0.02, map_seed=2), W.jet_flow(mach=1.5, re=2e4), 13)]
    grids = [jz.Grid(g, stream=stream).init(f, s) for g, f, s in cases]
    jz.jz_set_tiling(grids[0].h, 3)
    b = jz.Batch(grids, stream=stream)
    b.nsteps(5, cfl=0.5)
    stream.synchronize()
    for (gd, f, s), g in zip(cases, grids):
        o = oracle.Oracle(gd, f)
        Q = o.init(s)
        o.run(Q, 5, cfl=0.5)
        err = _rel_err(g.download(), o.inner(Q))
        assert err <= 1e-10, (gd["ni"], gd["nj"], gd["nk"], err)
        assert g.diagnostics()["time"] == pytest.approx(o.time, rel=1e-12)
    b.close()
