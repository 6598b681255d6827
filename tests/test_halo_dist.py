"""The rank-to-rank halo exchange of a partitioned grid (paper Section 4.1:
one partition per process; Section 4.3: two ghost layers of Q exchanged by
point-to-point messages at every stage), on CPU ranks over gloo.

Every rank holds its blocks as padded host arrays of a seeded global array
(the values a boundary pass would have left in the physical ghosts, NaN in
the exchange ghosts).  After ``HaloExchange.exchange`` every block, ghosts
included, must equal the global array bitwise: the interfaces are matched in
one global order, the directions are exchanged i, j, k (edge and corner
ghosts take values already received), faces between two blocks of one rank
need no message, and the rate maximum is taken over ranks.  The host block
adapter below mirrors the device buffer layout [v][layer][b][a]; the device
pack / unpack kernels and the stepping entry points are checked on the GPU
(tests/test_gpu_halo.py)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class HostBlock:
    """A block's three state copies as padded host arrays (5, nk+4, nj+4,
    ni+4); pack / unpack move the two layers of a face to / from a flat
    buffer in the device layout."""

    def __init__(self, arrays):
        import torch
        self.torch = torch
        self.A = arrays
        self.n = (arrays[0].shape[3] - 4, arrays[0].shape[2] - 4, arrays[0].shape[1] - 4)

    def _view(self, which, d, first):
        A, s = self.A[which], first + 2
        if d == 0:
            return A[:, :, :, s:s + 2].transpose(0, 3, 1, 2)   # [v][l][k][j]
        if d == 1:
            return A[:, :, s:s + 2, :].transpose(0, 2, 1, 3)   # [v][l][k][i]
        return A[:, s:s + 2, :, :]                             # [v][l][j][i]

    def pack(self, which, d, side):
        first = 0 if side == 0 else self.n[d] - 2
        return self.torch.from_numpy(np.ascontiguousarray(self._view(which, d, first)).reshape(-1))

    def recv_buffer(self, d, side):
        e = [self.n[x] + 4 for x in range(3) if x != d]
        return self.torch.empty(10 * e[0] * e[1], dtype=self.torch.float64)

    def unpack(self, which, d, side, buf):
        first = -2 if side == 0 else self.n[d]
        view = self._view(which, d, first)
        view[...] = buf.numpy().reshape(view.shape)


def _rank(rank, world, port, parts, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2003_09926_gb300 import halo
    from paper_2003_09926_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        desc = W.jet_grid(17, 11, 13)
        part = halo.Partition.even(desc, parts, world)
        rng = np.random.default_rng(5)
        G = [rng.standard_normal((5, 13 + 4, 11 + 4, 17 + 4)) for _ in range(3)]
        n = (17, 11, 13)
        blocks = {}
        for b in part.blocks_of(rank):
            o0, o1 = part.block(b)
            arrs = []
            for which in range(3):
                A = G[which][:, o0[2]:o1[2] + 5, o0[1]:o1[1] + 5, o0[0]:o1[0] + 5].copy()
                for d in range(3):
                    ax = 3 - d
                    if o0[d] > 0:  # exchange ghosts behind a low face: unknown before the exchange
                        A[(slice(None),) * ax + (slice(0, 2),)] = np.nan
                    if o1[d] < n[d] - 1:
                        A[(slice(None),) * ax + (slice(-2, None),)] = np.nan
                arrs.append(A)
            blocks[b] = HostBlock(arrs)
        ex = halo.HaloExchange(part, rank, blocks, halo.TorchTransport())
        for which in (0, 2, 1):
            ex.exchange(which)
        ok = True
        for b, blk in blocks.items():
            o0, o1 = part.block(b)
            for which in range(3):
                want = G[which][:, o0[2]:o1[2] + 5, o0[1]:o1[1] + 5, o0[0]:o1[0] + 5]
                ok = ok and bool(np.array_equal(blk.A[which], want))
        rate = torch.tensor([1.0 + 0.25 * rank], dtype=torch.float64)
        halo.TorchTransport().allreduce_max(rate)
        out.put((rank, ok, sorted(blocks), float(rate[0])))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,parts", [(2, (2, 1, 1)), (4, (2, 1, 2)), (2, (2, 1, 2)), (3, (1, 3, 2))])
def test_exchange_fills_every_ghost_bitwise(world, parts):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, parts, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    nblocks = parts[0] * parts[1] * parts[2]
    assert sorted(b for _, _, bs, _ in res for b in bs) == list(range(nblocks))
    for rank, ok, bs, rate in res:
        assert ok, (rank, bs)
        assert rate == 1.0 + 0.25 * (world - 1)


def test_partition_plan():
    sys.path.insert(0, ROOT)
    from paper_2003_09926_gb300 import halo
    from paper_2003_09926_gb300 import workloads as W
    part = halo.Partition.even(W.jet_grid(40, 24, 22), (2, 1, 3), world=4)
    assert len(part) == 6 and part.shape == (2, 1, 3)
    assert part.block(0) == ((0, 0, 0), (19, 23, 6)) and part.block(5) == ((20, 0, 15), (39, 23, 21))
    assert part.interfaces(0) == [(0, 1), (2, 3), (4, 5)]
    assert part.interfaces(1) == []
    assert part.interfaces(2) == [(0, 2), (1, 3), (2, 4), (3, 5)]
    assert part.blocks_of(1) == [1, 5] and part.owner(4) == 0
    assert halo.split_ranges(10, 3) == [(0, 2), (3, 6), (7, 9)]
    with pytest.raises(ValueError):
        halo.Partition(W.jet_grid(10, 8, 8), [[(0, 4), (6, 9)], [(0, 7)], [(0, 7)]])
    two = halo.Partition.even(W.jet_grid(20, 10, 10), (2, 1, 1), world=3)
    with pytest.raises(ValueError):  # rank 2 owns no block
        halo.HaloExchange(two, 2, {}, halo.LocalTransport())
    with pytest.raises(ValueError):  # blocks that are not the rank's
        halo.HaloExchange(two, 0, {1: None}, halo.LocalTransport())
