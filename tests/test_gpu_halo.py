"""The per-block entry points of a grid partitioned over ranks (jz_halo_pack
/ unpack, jz_block_rate / advance / stage) driven by halo.HaloExchange, with
every block in this process (the face buffers are unpacked straight from the
sender's; on several ranks they travel by point-to-point messages, whose
plan tests/test_halo_dist.py checks).  Paper Section 4.1-4.3: every block's
nodes must evolve bitwise as the same nodes of the undivided grid, and the
blocks share its time step."""
import numpy as np
import pytest

from paper_2003_09926_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09926_gb300 import build, halo, jz
    build.build()
    jz.lib()
    return jz, halo


@pytest.mark.parametrize("prec,parts", [(W.P64, (2, 1, 2)), (W.P32, (3, 2, 1)), (W.P32, (2, 2, 2))])
def test_ranked_blocks_step_like_the_whole_grid(mods, prec, parts):
    import torch
    jz, halo = mods
    grid = W.jet_grid(45, 26, 22, map_amp=0.04, map_seed=7, precision=prec)
    flow = W.jet_flow(re=3e4)
    stream = torch.cuda.Stream()
    whole = jz.Grid(grid, stream=stream).init(flow, 4)
    whole.nsteps(4, cfl=0.5)
    ref = whole.download()
    dref = whole.diagnostics()
    whole.close()
    part = halo.Partition.even(grid, parts, world=1)
    grids = halo.block_grids(part, 0, stream)
    for g in grids.values():
        g.init(flow, 4)
    ex = halo.HaloExchange(part, 0, {b: halo.DeviceBlock(g) for b, g in grids.items()}, halo.LocalTransport(),
                           stream=stream)
    for _ in range(4):
        ex.step(0.5)
    stream.synchronize()
    for b, g in grids.items():
        (i0, j0, k0), (i1, j1, k1) = part.block(b)
        np.testing.assert_array_equal(g.download(), ref[:, k0:k1 + 1, j0:j1 + 1, i0:i1 + 1], err_msg=f"block {b}")
        d = g.diagnostics()
        assert d["dt"] == dref["dt"] and d["time"] == dref["time"] and d["step"] == 4
        g.close()


def test_halo_entry_points_reject_bad_faces(mods):
    import torch
    jz, halo = mods
    grid = W.jet_grid(30, 20, 16, precision=W.P32)
    part = halo.Partition.even(grid, (2, 1, 1))
    g = halo.block_grids(part, 0, torch.cuda.Stream())[0]
    g.init(W.jet_flow(), 0)
    assert jz.jz_halo_bytes(g.h, 0) == 10 * (20 + 4) * (16 + 4) * 4
    buf = torch.empty(jz.jz_halo_bytes(g.h, 0), dtype=torch.uint8, device="cuda")
    jz.jz_halo_pack(g.h, 0, 0, 1, buf.data_ptr())  # the high i face is an exchange face
    for args in ((0, 0, 0), (0, 1, 1), (3, 0, 1), (0, 0, 2)):  # x- inflow, y+ far field, bad copy, bad side
        with pytest.raises(jz.JzError) as ei:
            jz.jz_halo_pack(g.h, *args, buf.data_ptr())
        assert ei.value.code == jz.JZ_EINVAL
    with pytest.raises(jz.JzError):
        jz.jz_block_stage(g.h, 5)
    with pytest.raises(jz.JzError):
        jz.jz_block_advance(g.h, 0.0)
    g.close()
