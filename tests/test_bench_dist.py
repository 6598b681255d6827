"""Multi-rank logic of bench.py on CPU ranks (gloo, world size 2): each rank
advances an independent grid, the job time is the maximum over ranks, and
the whole-job value counts every rank's points (weak scaling, no data-path
collective).  The reference arm prints from rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0, 25.0][rank]
    slowest = bench.reduce_max(torch, ms, world, "cpu")
    value = bench.weak_value(1000, 4, slowest, world)
    buf = io.StringIO()
    args = bench.argparse.Namespace(gpus=world, steps=1, warmup=0)
    if rank == 1:  # reference arm on a non-zero rank: no work, no output
        with redirect_stdout(buf):
            rc = bench.run_reference(args, rank, world)
        assert rc == 0 and buf.getvalue() == ""
    dist.barrier()
    out.put((rank, slowest, value))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_weak_value():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value in res:
        assert slowest == 25.0
        assert value == pytest.approx(2 * 1000 * 5 * 4 / 0.025 / 1e6)


def test_reference_arm_prints_one_line_on_rank0(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = bench.argparse.Namespace(gpus=1, steps=1, warmup=0)
    assert bench.run_reference(args, 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "Mpt-stage/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_is_silent_on_other_ranks(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = bench.argparse.Namespace(gpus=2, steps=1, warmup=0)
    assert bench.run_reference(args, 1, 2) == 0
    assert capsys.readouterr().out.strip() == ""
