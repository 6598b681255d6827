"""Blocks of one grid stepped as a block set (the paper's domain
decomposition with ghost exchange, Section 4.2, on one device): every block's
nodes must evolve bitwise as the same nodes of the whole grid stepped alone,
for splits along one, two and three directions, uneven block sizes, FP64 and
FP32, with the far-field, inflow and periodic boundary kinds present."""
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


def ranges(n, cuts):
    """[lo, hi] node ranges of a direction of n nodes cut before the given indices."""
    edges = [0] + list(cuts) + [n]
    return [(edges[a], edges[a + 1] - 1) for a in range(len(edges) - 1)]


def run_blocks(jz, grid, flow, seed, steps, cuts):
    import torch
    stream = torch.cuda.Stream()
    whole = jz.Grid(grid, stream=stream).init(flow, seed)
    whole.nsteps(steps, cfl=0.5)
    ref = whole.download()
    dref = whole.diagnostics()
    rs = [ranges(n, c) for n, c in zip((grid["ni"], grid["nj"], grid["nk"]), cuts)]
    blocks = []
    for ri in rs[0]:
        for rj in rs[1]:
            for rk in rs[2]:
                o0, o1 = (ri[0], rj[0], rk[0]), (ri[1], rj[1], rk[1])
                blocks.append(jz.Grid(grid, stream=stream, block=(o0, o1)).init(flow, seed))
    bs = jz.Batch(blocks, stream=stream, coupled=True)
    bs.nsteps(steps, cfl=0.5)
    stream.synchronize()
    for b in blocks:
        (i0, j0, k0), (i1, j1, k1) = b.block
        got = b.download()
        want = ref[:, k0:k1 + 1, j0:j1 + 1, i0:i1 + 1]
        np.testing.assert_array_equal(got, want, err_msg=f"block {b.block}")
        d = b.diagnostics()
        assert d["dt"] == dref["dt"] and d["time"] == dref["time"] and d["step"] == dref["step"]
    bs.close()
    for b in blocks:
        b.close()
    whole.close()
    return len(blocks)


@pytest.mark.parametrize("prec", [W.P64, W.P32])
def test_blocks_split_in_i_and_k_match_the_whole_grid(jz, prec):
    grid = W.jet_grid(48, 32, 32, map_amp=0.05, map_seed=3, precision=prec)
    assert run_blocks(jz, grid, W.jet_flow(), 2, 4, ([24], [], [16])) == 4


@pytest.mark.parametrize("prec", [W.P64, W.P32])
def test_blocks_uneven_split_in_three_directions(jz, prec):
    """Corner and edge ghosts take values exchanged in earlier directions; the
    blocks are of unequal size and smaller than one tile in some directions."""
    grid = W.jet_grid(45, 23, 19, map_amp=0.04, map_seed=7, precision=prec)
    assert run_blocks(jz, grid, W.jet_flow(re=2e4), 5, 3, ([13, 30], [11], [6, 12])) == 18


def test_blocks_with_a_periodic_direction(jz):
    """Periodic in k (not split), split in i and j."""
    grid = dict(W.jet_grid(40, 24, 12, map_amp=0.03, map_seed=2, precision=W.P32))
    grid["bc"] = [W.BC_INFLOW, W.BC_FARFIELD, W.BC_FARFIELD, W.BC_FARFIELD, W.BC_PERIODIC, W.BC_PERIODIC]
    assert run_blocks(jz, grid, W.jet_flow(), 1, 3, ([20], [12], [])) == 4


def test_block_sets_that_do_not_partition_the_grid_are_rejected(jz):
    import torch
    grid = W.jet_grid(40, 24, 16, precision=W.P32)
    stream = torch.cuda.Stream()
    a = jz.Grid(grid, stream=stream, block=((0, 0, 0), (19, 23, 15)))
    b = jz.Grid(grid, stream=stream, block=((18, 0, 0), (39, 23, 15)))  # overlaps a
    with pytest.raises(jz.JzError):
        jz.Batch([a, b], stream=stream, coupled=True)
    c = jz.Grid(grid, stream=stream, block=((20, 0, 0), (39, 11, 15)))  # half a face
    with pytest.raises(jz.JzError):
        jz.Batch([a, c], stream=stream, coupled=True)
    with pytest.raises(jz.JzError):  # a periodic direction cannot be split
        g = dict(grid, bc=[W.BC_INFLOW, W.BC_FARFIELD, W.BC_FARFIELD, W.BC_FARFIELD, W.BC_PERIODIC, W.BC_PERIODIC])
        jz.Grid(g, stream=stream, block=((0, 0, 0), (39, 23, 7)))
    with pytest.raises(jz.JzError):  # too thin along a split direction
        jz.Grid(grid, stream=stream, block=((0, 0, 0), (1, 23, 15)))


def test_p64_block_set_matches_the_oracle(jz):
    """Direct parity of the decomposed path (paper Section 4.2: partitioned
    domain, two-layer ghost exchange per stage): an FP64 block set split in
    i and k, advanced five steps with the whole grid's time step, reassembled
    and compared with the CPU oracle on the undivided grid, within 1e-10."""
    import torch

    import oracle
    grid = W.jet_grid(40, 24, 22, map_amp=0.04, map_seed=4)
    flow = W.jet_flow(re=5e4)
    stream = torch.cuda.Stream()
    blocks = []
    for ri in ranges(40, [17]):
        for rk in ranges(22, [9, 15]):
            blocks.append(jz.Grid(grid, stream=stream, block=((ri[0], 0, rk[0]), (ri[1], 23, rk[1]))).init(flow, 6))
    bs = jz.Batch(blocks, stream=stream, coupled=True)
    bs.nsteps(5, cfl=0.5)
    stream.synchronize()
    got = np.zeros((5, 22, 24, 40))
    for b in blocks:
        (i0, j0, k0), (i1, j1, k1) = b.block
        got[:, k0:k1 + 1, j0:j1 + 1, i0:i1 + 1] = b.download()
    o = oracle.Oracle(grid, flow)
    Q = o.init(6)
    o.run(Q, 5, cfl=0.5)
    ref = o.inner(Q)
    err = max(np.abs(got[v] - ref[v]).max() / np.abs(ref[v]).max() for v in range(5))
    assert err <= 1e-10, err
    bs.close()
    for b in blocks:
        b.close()
