"""The paper's cylindrical jet grid on the GPU (Section 3: centreline
singularity averaged azimuthally, superposed first and last azimuthal
points; Tab. mesh: 361 azimuthal points): parity with the FP64 oracle, the
invariants of the centreline and of the superposed plane, i-split blocks,
batches mixing cylinders and boxes, and the descriptor checks."""
import os

import numpy as np
import pytest

from paper_2003_09926_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jz():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09926_gb300 import build, jz as J
    build.build()
    J.lib()
    return J


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    return oracle


def rel_err(a, b):
    return max(np.abs(a[v] - b[v]).max() / np.abs(b[v]).max() for v in range(5))


def invariants(Q):
    """The last azimuthal plane repeats the first; centreline nodes away from
    the x faces are equal along the azimuth."""
    assert np.array_equal(Q[:, -1], Q[:, 0])
    assert np.array_equal(Q[:, :, 0, 1:-1], np.broadcast_to(Q[:, :1, 0, 1:-1], Q[:, :, 0, 1:-1].shape))


@pytest.mark.parametrize("shape,steps", [((24, 12, 33), 8), ((37, 19, 25), 5), ((20, 10, 361), 3)])
def test_cylinder_fp64_matches_oracle(jz, orc, shape, steps):
    grid = W.cyl_grid(*shape)
    flow = W.jet_flow(re=2e4)
    g = jz.Grid(grid).init(flow, 5)
    o = orc.Oracle(grid, flow)
    Q = o.init(5)
    np.testing.assert_allclose(g.download(), o.inner(Q), rtol=0, atol=1e-13)
    g.nsteps(steps, cfl=0.5)
    o.run(Q, steps, cfl=0.5)
    got = g.download()
    err = rel_err(got, o.inner(Q))
    assert err <= 1e-10, err
    invariants(got)
    d = g.diagnostics()
    assert abs(d["dt"] - o.last_dt) <= 1e-12 * o.last_dt
    np.testing.assert_allclose(d["sum"], o.diagnostics(Q)["sum"], rtol=1e-12)


@pytest.mark.parametrize("variant", [0, 2])
def test_cylinder_fp32_kernels_against_oracle(jz, orc, variant):
    """FP32 state and fluxes on the cylinder: the bounds of the box jet case
    (nodes at least 3 from the x and outer faces; the centreline and its
    neighbours included) after 10 steps."""
    grid = W.cyl_grid(40, 16, 33)
    flow = W.jet_flow(re=2e4)
    o = orc.Oracle(grid, flow)
    Q = o.init(2)
    o.run(Q, 10, cfl=0.5)
    ref = o.inner(Q)
    g = jz.Grid(dict(grid, precision=W.P32)).init(flow, 2)
    jz.jz_set_stage_variant(g.h, variant)
    g.nsteps(10, cfl=0.5)
    got = g.download()
    invariants(got)
    sel = (slice(None), slice(None), slice(0, -3), slice(3, -3))
    for v in range(5):
        e = np.abs(got[v][sel[1:]] - ref[v][sel[1:]]).max() / np.abs(ref[v]).max()
        assert e <= (2e-3 if v in (2, 3) else 5e-5), (variant, v, e)


@pytest.mark.parametrize("prec", [W.P64, W.P32])
def test_cylinder_blocks_split_in_i_match_the_whole_grid(jz, prec):
    import torch
    grid = W.cyl_grid(45, 12, 25, precision=prec)
    flow = W.jet_flow()
    stream = torch.cuda.Stream()
    whole = jz.Grid(grid, stream=stream).init(flow, 3)
    whole.nsteps(4, cfl=0.5)
    ref = whole.download()
    cuts = [(0, 14), (15, 31), (32, 44)]
    blocks = [jz.Grid(grid, stream=stream, block=((a, 0, 0), (b, 11, 24))).init(flow, 3) for a, b in cuts]
    bs = jz.Batch(blocks, stream=stream, coupled=True)
    bs.nsteps(4, cfl=0.5)
    stream.synchronize()
    for (a, b), blk in zip(cuts, blocks):
        np.testing.assert_array_equal(blk.download(), ref[:, :, :, a:b + 1])
    bs.close()
    with pytest.raises(jz.JzError):  # a cylinder splits in i only
        jz.Grid(grid, stream=stream, block=((0, 0, 0), (44, 5, 24)))


def test_batch_of_cylinders_and_boxes_equals_grids_alone(jz):
    import torch
    stream = torch.cuda.Stream()
    cases = [(W.cyl_grid(30, 10, 21, precision=W.P32), 1), (W.jet_grid(33, 17, 19, precision=W.P32), 2),
             (W.cyl_grid(17, 9, 13, precision=W.P32), 3)]
    grids = [jz.Grid(g, stream=stream).init(W.jet_flow(), s) for g, s in cases]
    b = jz.Batch(grids, stream=stream)
    b.nsteps(5, cfl=0.5)
    stream.synchronize()
    for (g, s), bg in zip(cases, grids):
        alone = jz.Grid(g).init(W.jet_flow(), s)
        alone.nsteps(5, cfl=0.5)
        np.testing.assert_array_equal(bg.download(), alone.download())
    b.close()


def test_cylinder_descriptor_checks(jz):
    good = W.cyl_grid(16, 8, 13)
    jz.Grid(good).close()
    bad = [dict(good, nk=14),                                  # nk - 1 odd
           dict(good, map_amp=0.01),                           # no mapping on a cylinder
           dict(good, lo=[0.0, 0.5, 0.0]),                     # radius starts at 0
           dict(good, bc=[W.BC_INFLOW, W.BC_FARFIELD, W.BC_FARFIELD, W.BC_FARFIELD, W.BC_PERIODIC, W.BC_PERIODIC]),
           dict(W.jet_grid(16, 8, 13), bc=[W.BC_INFLOW, W.BC_FARFIELD, W.BC_AXIS, W.BC_FARFIELD,
                                           W.BC_FARFIELD, W.BC_FARFIELD]),  # axis on a box
           dict(good, geom=7)]
    for d in bad:
        with pytest.raises(jz.JzError):
            jz.Grid(d)


@pytest.mark.parametrize("shape", [(3, 4, 5), (5, 4, 9)])
def test_smallest_cylinders_match_oracle(jz, orc, shape):
    """The smallest cylinders the descriptor allows (nj = 4: one radial line
    between the centreline and the far field; nk = 5: four azimuthal
    intervals)."""
    grid = W.cyl_grid(*shape, length=2.0, radius=1.5)
    flow = W.jet_flow(re=5e3)
    g = jz.Grid(grid).init(flow, 1)
    o = orc.Oracle(grid, flow)
    Q = o.init(1)
    g.nsteps(4, cfl=0.5)
    o.run(Q, 4, cfl=0.5)
    got = g.download()
    assert rel_err(got, o.inner(Q)) <= 1e-10
    invariants(got)


def test_cylinder_with_vreman_and_fp64_state(jz, orc):
    """The options combine: Vreman eddy viscosity on the cylinder in FP64
    (against the oracle) and with the FP64-state FP32 mode (FP32 bounds)."""
    grid = W.cyl_grid(30, 12, 25)
    flow = W.jet_flow(re=5e3, sgs=W.SGS_VREMAN)
    o = orc.Oracle(grid, flow)
    Q = o.init(6)
    o.run(Q, 6, cfl=0.5)
    ref = o.inner(Q)
    g = jz.Grid(grid).init(flow, 6)
    g.nsteps(6, cfl=0.5)
    assert rel_err(g.download(), ref) <= 1e-10
    g32 = jz.Grid(dict(grid, precision=W.P32_S64)).init(flow, 6)
    g32.nsteps(6, cfl=0.5)
    got = g32.download()
    invariants(got)
    sel = (slice(None), slice(0, -3), slice(3, -3))
    for v in range(5):
        e = np.abs(got[v][sel] - ref[v][sel]).max() / np.abs(ref[v]).max()
        assert e <= (2e-3 if v in (2, 3) else 5e-5), (v, e)


def seq_mean(ring):
    """The mean of one azimuthal ring summed in azimuthal order in FP64."""
    s = 0.0
    for x in ring:
        s += float(x)
    return s / len(ring)


def check_centreline_sequential(Q, grid, prec):
    P = grid["nk"] - 1
    for v in range(5):
        for i in range(1, grid["ni"] - 1):  # the x faces own their centreline nodes
            m = seq_mean(Q[v, :P, 1, i])
            want = float(np.float32(m)) if prec != W.P64 else m
            assert np.all(Q[v, :, 0, i] == want), (v, i)


@pytest.mark.parametrize("prec", [W.P64, W.P32])
def test_centreline_is_the_sequential_fp64_mean(jz, prec):
    """Section 4.3: the centreline average is formed sequentially so that a
    parallel run reproduces the serial one bit for bit.  Every centreline
    node away from the x faces must be bitwise the FP64 mean of its j = 1
    ring summed in azimuthal order, rounded to the state's type: after steps
    of the jet, and for uploaded rings that force the FP32 kernel off its
    exact integer sum (values 2^40 apart, a NaN-free ring with exact
    cancellation, all-zero rings, subnormal FP32 values)."""
    grid = W.cyl_grid(20, 10, 65, precision=prec)
    g = jz.Grid(grid).init(W.jet_flow(re=2e4), 3)
    g.nsteps(3, cfl=0.5)
    Q = g.download()
    check_centreline_sequential(Q, grid, prec)
    rng = np.random.default_rng(11)
    P = grid["nk"] - 1
    Q = Q.copy()
    ring = Q[1, :P, 1, 4]
    ring[:] = rng.uniform(0.5, 1.5, P)
    ring[::7] = 1e-12 * rng.uniform(1, 2, ring[::7].size)  # unit in the last place far below the sum: rounding
    Q[2, :P, 1, 5] = np.where(np.arange(P) % 2 == 0, 0.75, -0.75)  # exact cancellation
    Q[3, :P, 1, 6] = 0.0
    Q[2, :P, 1, 7] = 1e-40 * rng.uniform(-1, 1, P)  # subnormal in FP32
    Q[3, :P, 1, 8] = rng.uniform(-1, 1, P) * 2.0 ** rng.integers(-30, 30, P)  # wide exponent spread
    Q[:, P] = Q[:, 0]
    g.upload(Q)
    got = g.download()
    check_centreline_sequential(got, grid, prec)
    g.close()
