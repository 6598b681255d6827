"""Host-side logic of the serving loop, on the CPU with a fake device
backend: admission by budget, slice selection (oldest first or least
remaining work first) and request cancellation.  The fake grids count the
steps they are advanced; nothing here touches a GPU."""
import threading
import time

import pytest

from paper_2003_09926_gb300 import serve
from paper_2003_09926_gb300 import workloads as W


class FakeGrid:
    def __init__(self, log, desc, seed):
        self.log, self.desc, self.seed = log, desc, seed
        self.steps = 0
        self.closed = False
        log.append(("create", seed))

    def nsteps(self, n, cfl=0.5):
        assert not self.closed
        self.steps += n

    def diagnostics(self, allow_nonfinite=False):
        return {"step": self.steps}

    def download(self):
        return self.steps

    def close(self):
        self.closed = True
        self.log.append(("close", self.seed))

    def set_stream(self, stream):
        self.log.append(("stream", self.seed, stream))
        self.stream = stream


class FakeBatch:
    def __init__(self, grids):
        self.grids = grids
        self.closed = False

    def nsteps(self, n, cfl):
        assert not self.closed
        for g in self.grids:
            g.nsteps(n, cfl)

    def close(self):
        self.closed = True


class FakeBackend:
    def __init__(self, slice_delay=0.0):
        self.log = []
        self.grids = {}
        self.slice_delay = slice_delay

    def grid_bytes(self, desc):
        return desc["ni"] * desc["nj"] * desc["nk"]

    def grid(self, desc, flow, seed, kc, stream=None):
        g = FakeGrid(self.log, desc, seed)
        g.stream = stream
        self.grids[seed] = g
        return g

    def priority_streams(self, n):
        return [f"s{i}" for i in range(n)]

    def done(self, ev):
        return True

    def batch(self, grids):
        return FakeBatch(grids)

    def synchronize(self):
        if self.slice_delay:
            time.sleep(self.slice_delay)
        self.log.append(("sync", None))

    def mark(self, stream=None):
        return object()

    def wait(self, ev):
        if self.slice_delay:
            time.sleep(self.slice_delay)


def _req(rid, n, steps, arrival=0.0, cancel_at=None):
    return serve.Request(rid, W.jet_grid(n, n, n, precision=W.P32), W.jet_flow(), rid, steps, arrival, cancel_at)


def test_cancel_before_admission_never_creates_the_grid():
    be = FakeBackend()
    reqs = [_req(0, 10, 20), _req(1, 10, 20, arrival=0.05, cancel_at=0.0)]
    res = serve.Server(10 ** 6, slice_steps=5, backend=be).run(reqs)
    assert res[0].status == "done" and res[0].diag["step"] == 20
    assert res[1].status == "cancelled"
    assert ("create", 1) not in be.log


def test_cancel_of_a_resident_case_frees_its_memory():
    """Budget for one case: case 1 waits until case 0 is cancelled part way,
    then is admitted and completes; case 0 stops short of its steps and its
    grid is closed."""
    be = FakeBackend(slice_delay=0.01)
    reqs = [_req(0, 10, 10 ** 6, cancel_at=0.05), _req(1, 10, 30, arrival=0.01)]
    srv = serve.Server(1000, slice_steps=5, backend=be)
    res = srv.run(reqs)
    assert res[0].status == "cancelled" and res[0].diag is None
    assert 0 < be.grids[0].steps < 10 ** 6 and be.grids[0].closed
    assert res[1].status == "done" and res[1].diag["step"] == 30
    assert be.log.index(("close", 0)) < be.log.index(("create", 1))
    assert srv.peak_bytes == 1000


def test_cancel_from_another_thread():
    be = FakeBackend(slice_delay=0.005)
    reqs = [_req(0, 8, 10 ** 6), _req(1, 8, 40)]
    srv = serve.Server(10 ** 6, slice_steps=2, backend=be, fill_points=1, order="arrival")
    t = threading.Timer(0.05, srv.cancel, args=(0,))
    t.start()
    res = srv.run(reqs)
    t.join()
    assert res[0].status == "cancelled" and res[1].status == "done" and res[1].diag["step"] == 40
    assert all(g.closed for g in be.grids.values())
    s = serve.summarize(res)
    assert s["completed"] == 1 and s["rejected"] == 1


def test_least_remaining_work_first():
    """With room for one case per slice, least-remaining-work order finishes
    the small late case before the large early one; oldest-first does the
    opposite."""
    reqs = [_req(0, 20, 60), _req(1, 10, 10)]
    fin = {}
    for order in ("remaining", "arrival"):
        be = FakeBackend()
        res = serve.Server(10 ** 6, slice_steps=5, backend=be, fill_points=1, order=order).run(reqs)
        assert all(r.status == "done" for r in res)
        fin[order] = [r.finished for r in res]
    assert fin["remaining"][1] < fin["remaining"][0]
    assert fin["arrival"][0] < fin["arrival"][1]


def test_head_order_keeps_the_oldest_case_moving():
    """'head': the oldest case is always in the slice; the fill comes from
    the least remaining work."""
    mk = lambda rid, n, left, arr: {"req": _req(rid, n, 100, arr), "left": left}  # noqa: E731
    res = [mk(0, 20, 50, 0.0), mk(1, 10, 50, 1.0), mk(2, 30, 1, 2.0)]
    assert [c["req"].rid for c in serve.select_cases(res, 6000, "head")] == [0, 2]
    assert [c["req"].rid for c in serve.select_cases(res, 5000, "head")] == [0]
    reqs = [_req(0, 20, 60), _req(1, 10, 10, arrival=0.0)]
    be = FakeBackend()
    out = serve.Server(10 ** 6, slice_steps=5, backend=be, fill_points=1, order="head").run(reqs)
    assert [r.diag["step"] for r in out] == [60, 10]
    assert out[0].finished < out[1].finished  # fill 1: the oldest runs alone, first


def test_results_wait_for_their_slice():
    """Slices are pipelined, but a case's result is read only after the
    device has finished it (a synchronisation precedes every retirement)."""
    be = FakeBackend()
    reqs = [_req(0, 10, 30), _req(1, 12, 45)]
    serve.Server(10 ** 6, slice_steps=10, backend=be, fill_points=10 ** 9).run(reqs)
    for seed in (0, 1):
        i = be.log.index(("close", seed))
        assert ("sync", None) in be.log[:i]


def test_select_cases_orders():
    mk = lambda rid, n, left, arr: {"req": _req(rid, n, 100, arr), "left": left}  # noqa: E731
    res = [mk(0, 20, 50, 0.0), mk(1, 10, 50, 1.0), mk(2, 30, 1, 2.0)]
    # updated points: 18^3 = 5832, 8^3 = 512, 28^3 = 21952; remaining work 291600, 25600, 21952
    assert [c["req"].rid for c in serve.select_cases(res, 6000, "remaining")] == [2]
    assert [c["req"].rid for c in serve.select_cases(res, 30000, "remaining")] == [2, 1, 0]
    assert [c["req"].rid for c in serve.select_cases(res, 6000, "arrival")] == [0, 1]
    assert len(serve.select_cases(res, None)) == 3
    with pytest.raises(ValueError):
        serve.select_cases(res, 10, "random")


def test_priority_server_ranks_streams_by_arrival():
    """The oldest resident case always holds the highest-priority stream;
    when it finishes, the next one moves up (at a chunk boundary)."""
    be = FakeBackend()
    reqs = [_req(0, 10, 40), _req(1, 10, 100), _req(2, 10, 60)]
    srv = serve.PriorityServer(10 ** 6, max_running=3, chunk_steps=10, backend=be, fill_ratio=None)
    res = srv.run(reqs)
    assert all(r.status == "done" for r in res) and [r.diag["step"] for r in res] == [40, 100, 60]
    assert be.grids[0].stream == "s0"
    moves = [e for e in be.log if e[0] == "stream"]
    # case 1 moves to s0 after case 0 retires; case 2 to s1, then s0 after case 1... or retires first
    assert ("stream", 1, "s0") in moves and ("stream", 2, "s1") in moves
    assert be.log.index(("close", 0)) < be.log.index(("stream", 1, "s0"))
    assert srv.chunks == 4 + 10 + 6


def test_priority_server_budget_slots_and_cancel():
    be = FakeBackend(slice_delay=0.0)
    reqs = [_req(0, 10, 10 ** 5, cancel_at=0.02), _req(1, 10, 30), _req(2, 10, 20, arrival=0.01)]
    srv = serve.PriorityServer(1000, max_running=4, chunk_steps=5, backend=be)  # memory for one case
    res = srv.run(reqs)
    assert res[0].status == "cancelled" and be.grids[0].closed
    assert res[1].status == "done" and res[2].status == "done"
    assert srv.peak_bytes == 1000
    assert be.log.index(("close", 0)) < be.log.index(("create", 1)) < be.log.index(("create", 2))


def test_priority_server_fills_only_with_small_work():
    """With fill_ratio, a case joins the resident oldest one only while its
    work is at most fill_ratio times the oldest's remaining work; a larger
    one waits (admission stays in arrival order, so the cases behind it
    wait too) until the oldest has retired."""
    be = FakeBackend()
    # case 0: 20^3 nodes x 200 steps; case 1: 10^3 x 40 (small: joins at
    # once); case 2: 20^3 x 200 (large: waits for case 0)
    reqs = [_req(0, 20, 200), _req(1, 10, 40), _req(2, 20, 200)]
    srv = serve.PriorityServer(10 ** 9, max_running=2, chunk_steps=20, backend=be, fill_ratio=0.25)
    res = srv.run(reqs)
    assert all(r.status == "done" for r in res)
    log = be.log
    assert log.index(("create", 1)) < log.index(("close", 0))  # filled in beside case 0
    assert log.index(("close", 0)) < log.index(("create", 2))  # held until case 0 retired
    # without the limit, the second slot takes case 2 as soon as case 1 retires
    be2 = FakeBackend()
    serve.PriorityServer(10 ** 9, max_running=2, chunk_steps=20, backend=be2, fill_ratio=None).run(reqs)
    assert be2.log.index(("create", 2)) < be2.log.index(("close", 0))
