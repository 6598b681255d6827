"""A grid partitioned over ranks: blocks, their two-layer halo exchange and
the combined time step.

Paper: arXiv 2003.09926, Section 4.1 (the domain is partitioned and every
process owns one partition), Section 4.3 (the two ghost layers of Q are
exchanged with the neighbouring partitions by non-blocking point-to-point
messages at every Runge-Kutta stage) and Section 4.2, Fig. jazzy (where the
exchanges sit in the stage sequence).  The time step of the CFL condition is
one value for the whole grid: every block's largest stable-step rate is
combined by a maximum over ranks.

Layout of the work: the grid is cut into a tensor product of node ranges
(``Partition``); a rank owns some blocks (``jz_block_create`` on its GPU) and
steps them with the per-block entry points of the C library
(``jz_block_rate``, ``jz_block_advance``, ``jz_block_stage``).  Between
stages, ``HaloExchange.exchange`` packs the two node layers of every
exchange face into a contiguous device buffer (``jz_halo_pack``), moves the
buffers with point-to-point sends and receives (``torch.distributed``: NCCL
for device buffers; no collective on the data path), and unpacks them into
the neighbours' ghost layers (``jz_halo_unpack``), direction by direction in
the order i, j, k over the padded extents of the other directions, so that
edge and corner ghosts take values already exchanged.  Every interface is
visited in one global order on every rank, so the messages between two
ranks match in order whatever the backend.  Blocks of one rank exchange
through the same plan with in-process copies (``LocalTransport``).

The arithmetic per node is that of the whole grid, so a partitioned run is
bitwise the undivided one.
"""
from __future__ import annotations

import contextlib

from . import jz

# output state copy of Runge-Kutta stage l (0 = Q0, 1 = QA, 2 = QB)
STAGE_OUT = (1, 2, 1, 2, 0)


def split_ranges(n: int, parts: int) -> list[tuple[int, int]]:
    """Cut n nodes into `parts` contiguous [lo, hi] ranges of near-equal size."""
    if not 1 <= parts <= n:
        raise ValueError(f"cannot cut {n} nodes into {parts} parts")
    edges = [round(p * n / parts) for p in range(parts + 1)]
    return [(edges[p], edges[p + 1] - 1) for p in range(parts)]


class Partition:
    """Blocks of a grid as a tensor product of node ranges per direction.

    ranges: three lists of inclusive (lo, hi) node ranges covering 0..n-1 in
    order (i, j, k).  Block b = (bi, bj, bk) has index bi + Pi (bj + Pj bk).
    owner: block index -> rank (default: block index modulo world)."""

    def __init__(self, desc: dict, ranges, world: int = 1, owner=None):
        self.desc = dict(desc)
        self.ranges = [list(r) for r in ranges]
        n = (desc["ni"], desc["nj"], desc["nk"])
        for d in range(3):
            r = self.ranges[d]
            if r[0][0] != 0 or r[-1][1] != n[d] - 1 or any(r[p][1] + 1 != r[p + 1][0] for p in range(len(r) - 1)):
                raise ValueError(f"ranges of direction {d} do not cover 0..{n[d] - 1} in order")
        self.shape = tuple(len(r) for r in self.ranges)
        self.world = world
        self._owner = owner if owner is not None else (lambda b: b % world)

    @classmethod
    def even(cls, desc: dict, parts, world: int = 1, owner=None) -> "Partition":
        n = (desc["ni"], desc["nj"], desc["nk"])
        return cls(desc, [split_ranges(n[d], parts[d]) for d in range(3)], world, owner)

    def __len__(self):
        return self.shape[0] * self.shape[1] * self.shape[2]

    def coords(self, b: int) -> tuple[int, int, int]:
        pi, pj, _ = self.shape
        return b % pi, (b // pi) % pj, b // (pi * pj)

    def index(self, c) -> int:
        pi, pj, _ = self.shape
        return c[0] + pi * (c[1] + pj * c[2])

    def block(self, b: int):
        """(o0, o1): the block's first and last global node per direction."""
        c = self.coords(b)
        return (tuple(self.ranges[d][c[d]][0] for d in range(3)), tuple(self.ranges[d][c[d]][1] for d in range(3)))

    def owner(self, b: int) -> int:
        return int(self._owner(b))

    def blocks_of(self, rank: int) -> list[int]:
        return [b for b in range(len(self)) if self.owner(b) == rank]

    def interfaces(self, d: int) -> list[tuple[int, int]]:
        """(a, b) pairs whose high face in direction d touches b's low face,
        in one global order (by a)."""
        out = []
        for b in range(len(self)):
            c = list(self.coords(b))
            if c[d] + 1 < self.shape[d]:
                c[d] += 1
                out.append((b, self.index(c)))
        return out


class DeviceBlock:
    """A block on this rank's GPU (a ``jz.Grid`` created with ``block=``) and
    its face buffers (device memory from PyTorch, allocated once)."""

    def __init__(self, grid: "jz.Grid"):
        import torch
        self.torch = torch
        self.grid = grid
        self.bufs = {}

    def buffer(self, d: int, side: int, kind: str):
        key = (d, side, kind)
        if key not in self.bufs:
            nbytes = jz.jz_halo_bytes(self.grid.h, d)
            self.bufs[key] = self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.grid.device)
        return self.bufs[key]

    def pack(self, which: int, d: int, side: int):
        buf = self.buffer(d, side, "send")
        jz.jz_halo_pack(self.grid.h, which, d, side, buf.data_ptr())
        return buf

    def unpack(self, which: int, d: int, side: int, buf) -> None:
        jz.jz_halo_unpack(self.grid.h, which, d, side, buf.data_ptr())

    def recv_buffer(self, d: int, side: int):
        return self.buffer(d, side, "recv")

    def rate(self):
        """Enqueue the block's rate; a one-element FP64 device tensor viewing it."""
        ptr = jz.jz_block_rate(self.grid.h)
        return self.torch.as_tensor(_DeviceScalar(ptr), device=self.grid.device)

    def advance(self, cfl: float) -> None:
        jz.jz_block_advance(self.grid.h, cfl)

    def stage(self, l: int) -> None:
        jz.jz_block_stage(self.grid.h, l)


class _DeviceScalar:
    """One FP64 value in device memory, exposed to PyTorch without a copy."""

    def __init__(self, ptr: int):
        self.__cuda_array_interface__ = {"shape": (1,), "typestr": "<f8", "data": (int(ptr), False), "version": 2}


class TorchTransport:
    """Point-to-point messages and the rate maximum through torch.distributed
    (NCCL for device buffers, gloo for host buffers)."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist

    def run(self, ops) -> None:
        """ops: ("send" | "recv", tensor, peer rank, tag), posted together."""
        if not ops:
            return
        p2p = [self.dist.P2POp(self.dist.isend if kind == "send" else self.dist.irecv, t, peer, tag=tag)
               for kind, t, peer, tag in ops]
        for req in self.dist.batch_isend_irecv(p2p):
            req.wait()

    def allreduce_max(self, t) -> None:
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)


class LocalTransport:
    """One process owns every block: no messages leave it (faces between two
    owned blocks are unpacked straight from the sender's buffer) and the
    rate maximum over ranks is the local one."""

    def run(self, ops) -> None:
        if ops:
            raise RuntimeError("local transport: a face has a neighbour on another rank")

    def allreduce_max(self, t) -> None:
        pass


class HaloExchange:
    """Exchange and stepping of the blocks this rank owns.

    blocks: block index -> adapter with pack(which, d, side) -> buffer,
    recv_buffer(d, side), unpack(which, d, side, buffer) and, for stepping,
    rate(), advance(cfl), stage(l) (``DeviceBlock``).  stream: the CUDA
    stream (torch.cuda.Stream) every owned block was created on; PyTorch's
    work (messages, the rate maximum) is issued on it, so it is ordered with
    the library's kernels."""

    def __init__(self, part: Partition, rank: int, blocks: dict, transport, stream=None):
        self.part = part
        self.rank = rank
        self.blocks = dict(blocks)
        self.transport = transport
        self.stream = stream
        mine = set(part.blocks_of(rank))
        if set(self.blocks) != mine:
            raise ValueError(f"rank {rank} owns blocks {sorted(mine)}, given {sorted(self.blocks)}")
        if not mine:
            raise ValueError(f"rank {rank} owns no block of the partition (every rank needs one)")

    def _on_stream(self):
        if self.stream is None:
            return contextlib.nullcontext()
        import torch
        return torch.cuda.stream(self.stream)

    def exchange(self, which: int) -> None:
        """Fill the exchange ghosts of state copy `which` of every owned block."""
        with self._on_stream():
            self._exchange(which)

    def _exchange(self, which: int) -> None:
        for d in range(3):
            ops, unpacks = [], []
            for q, (a, b) in enumerate(self.part.interfaces(d)):
                tag_up, tag_down = 2 * (d * len(self.part) + q), 2 * (d * len(self.part) + q) + 1
                if a in self.blocks and b in self.blocks:  # both here: no message
                    unpacks.append((self.blocks[b], d, 0, self.blocks[a].pack(which, d, 1)))
                    unpacks.append((self.blocks[a], d, 1, self.blocks[b].pack(which, d, 0)))
                    continue
                if a in self.blocks:  # a's high face (side 1) <-> b's low face
                    blk = self.blocks[a]
                    ops.append(("send", blk.pack(which, d, 1), self.part.owner(b), tag_up))
                    rbuf = blk.recv_buffer(d, 1)
                    ops.append(("recv", rbuf, self.part.owner(b), tag_down))
                    unpacks.append((blk, d, 1, rbuf))
                if b in self.blocks:
                    blk = self.blocks[b]
                    rbuf = blk.recv_buffer(d, 0)
                    ops.append(("recv", rbuf, self.part.owner(a), tag_up))
                    ops.append(("send", blk.pack(which, d, 0), self.part.owner(a), tag_down))
                    unpacks.append((blk, d, 0, rbuf))
            self.transport.run(ops)
            for blk, dd, side, rbuf in unpacks:
                blk.unpack(which, dd, side, rbuf)

    def step(self, cfl: float) -> None:
        """One time step of every owned block (the sequence of jz_block_*)."""
        with self._on_stream():
            self._step(cfl)

    def _step(self, cfl: float) -> None:
        self._exchange(0)
        rates = [blk.rate() for blk in self.blocks.values()]
        m = rates[0].clone()
        for r in rates[1:]:
            m = m.maximum(r)
        self.transport.allreduce_max(m)
        for r in rates:
            r.copy_(m)
        for blk in self.blocks.values():
            blk.advance(cfl)
        for l in range(5):
            for blk in self.blocks.values():
                blk.stage(l)
            if l < 4:
                self._exchange(STAGE_OUT[l])


def block_grids(part: Partition, rank: int, stream, device: int = 0) -> dict:
    """Create this rank's blocks on its GPU: block index -> ``jz.Grid``."""
    return {b: jz.Grid(part.desc, stream=stream, device=device, block=part.block(b)) for b in part.blocks_of(rank)}


__all__ = ["Partition", "DeviceBlock", "TorchTransport", "LocalTransport", "HaloExchange", "block_grids",
           "split_ranges", "STAGE_OUT"]
