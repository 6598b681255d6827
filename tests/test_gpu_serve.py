"""Continuous batching: cases arriving while others run are admitted as
memory frees up (HBM budget), advance together in time slices, and each
case's final state is bitwise the one it reaches when run alone."""
import numpy as np
import pytest

from paper_2003_09926_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09926_gb300 import build, jz, serve
    build.build()
    jz.lib()
    return jz, serve


def _trace(serve):
    shapes = [(40, 24, 20), (33, 17, 19), (24, 24, 24), (20, 40, 12), (48, 16, 24), (30, 20, 16)]
    steps = [12, 7, 23, 9, 15, 11]
    arrivals = [0.0, 0.0, 0.02, 0.05, 0.05, 0.1]
    reqs = []
    for i, (sh, n, t) in enumerate(zip(shapes, steps, arrivals)):
        flow = W.jet_flow(mach=1.2 + 0.1 * i, re=5e5 + 2e5 * i)
        reqs.append(serve.Request(i, W.jet_grid(*sh, map_amp=0.02, map_seed=i, precision=W.P32), flow, 50 + i, n,
                                  t))
    return reqs


def test_results_same_alone_and_in_the_mix(mods):
    jz, serve = mods
    reqs = _trace(serve)
    sizes = sorted(jz.jz_grid_bytes(r.grid) for r in reqs)
    budget = sizes[-1] + sizes[-2] + sizes[-3]  # at most about three cases resident
    srv = serve.Server(budget, slice_steps=5, keep_state=True)
    res = srv.run(reqs)
    assert all(r.status == "done" for r in res)
    assert srv.peak_bytes <= budget and srv.slices > 3
    for r, q in zip(res, reqs):
        alone = jz.Grid(q.grid).init(q.flow, q.seed)
        alone.nsteps(q.steps, cfl=0.5)
        np.testing.assert_array_equal(r.state, alone.download())
        assert r.diag["step"] == q.steps and r.latency > 0
        alone.close()
    s = serve.summarize(res)
    assert s["completed"] == 6 and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_over_budget_request_rejected(mods):
    jz, serve = mods
    reqs = _trace(serve)[:3]
    need = jz.jz_grid_bytes(reqs[0].grid)
    srv = serve.Server(need - 1, slice_steps=4)
    res = srv.run(reqs)
    assert res[0].status.startswith("rejected")
    assert all(r.status == "done" for r in res[1:] if jz.jz_grid_bytes(reqs[r.rid].grid) < need)


def test_served_p64_cases_match_the_oracle(mods):
    """Direct parity of the serving path: FP64 cases arriving at different
    times, served under a budget that holds two of them, advanced in
    slices mixed with each other, are each within 1e-10 of the CPU oracle
    run on that case alone."""
    import oracle
    jz, serve = mods
    shapes = [(30, 20, 16), (24, 18, 20), (36, 16, 14), (20, 20, 20)]
    reqs = []
    for i, sh in enumerate(shapes):
        flow = W.jet_flow(mach=1.3 + 0.15 * i, re=4e5 * (i + 1))
        reqs.append(serve.Request(i, W.jet_grid(*sh, map_amp=0.02 * (i % 2), map_seed=i, precision=W.P64), flow,
                                  70 + i, 6 + 2 * i, 0.01 * i))
    sizes = sorted(jz.jz_grid_bytes(r.grid) for r in reqs)
    srv = serve.Server(sizes[-1] + sizes[-2], slice_steps=3, keep_state=True)
    res = srv.run(reqs)
    assert all(r.status == "done" for r in res) and srv.slices >= 4
    for r, q in zip(res, reqs):
        o = oracle.Oracle(q.grid, q.flow)
        Q = o.init(q.seed)
        o.run(Q, q.steps, cfl=0.5)
        ref = o.inner(Q)
        err = max(np.abs(r.state[v] - ref[v]).max() / np.abs(ref[v]).max() for v in range(5))
        assert err <= 1e-10, (q.rid, err)


def test_priority_server_results_same_alone_and_in_the_mix(mods):
    """Prioritised streams: cases overlapping on the device (the oldest on
    the highest-priority stream, moved up as older cases finish) each end
    bitwise in the state they reach alone."""
    jz, serve = mods
    reqs = _trace(serve)
    sizes = sorted(jz.jz_grid_bytes(r.grid) for r in reqs)
    srv = serve.PriorityServer(sizes[-1] + sizes[-2] + sizes[-3], max_running=3, chunk_steps=4, keep_state=True,
                               fill_ratio=None)  # every case may overlap the oldest
    res = srv.run(reqs)
    assert all(r.status == "done" for r in res) and srv.chunks >= sum((q.steps + 3) // 4 for q in reqs)
    for r, q in zip(res, reqs):
        alone = jz.Grid(q.grid).init(q.flow, q.seed)
        alone.nsteps(q.steps, cfl=0.5)
        np.testing.assert_array_equal(r.state, alone.download())
        assert r.diag["step"] == q.steps
        alone.close()
