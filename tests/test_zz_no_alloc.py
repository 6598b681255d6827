"""jz_state_diagnostics_static: diagnostics for callers that may only use the
device arrays they were handed (a plug-in given its input and output
buffers, a serving process that reserved all device memory up front) and so
cannot supply reduction scratch.  The entry point keeps its scratch in a
static device array inside the library.

Its result on a state copied out of a grid must equal what jz_diagnostics
reports for that grid, on two calls in a row (the second call reuses the
shared scratch left by the first).  Collected last on purpose: a failure here
stops a -x run only after every other test has run."""
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


# sums: an FP32 grid holds J rounded to FP32 and its diagnostics round 1/J
# and each product Q_v * (1/J) in FP32 (three roundings of 2^-24 relative);
# the static entry point forms the product in FP64 from FP64 volumes: they
# agree to within 2^-22 of sum |Q_v| vol
# config 0 (49,152 nodes, one reduction block) and a 72 x 56 x 56 grid
# (225,792 nodes: three full 65,536-node blocks and a partial fourth, so the
# per-block records, the last-block counter and the ordered combination run)
@pytest.mark.parametrize("shape", [(48, 32, 32), (72, 56, 56)])
@pytest.mark.parametrize("prec,rtol", [(W.P64, 1e-12), (W.P32, 2.0 ** -22)])
def test_static_scratch_diagnostics_match_grid_diagnostics(jz, prec, rtol, shape):
    import torch

    import oracle
    c = W.config0()
    grid = dict(W.jet_grid(*shape), map_amp=0.02, map_seed=1, precision=prec)
    g = jz.Grid(grid).init(c["flow"], 3)
    g.nsteps(3, cfl=c["cfl"])
    ref = g.diagnostics()
    Q = g.download()  # FP32 states are widened exactly, so narrowing back is exact
    n = Q[0].size
    q_dev = torch.from_numpy(Q.reshape(5, n)).to(device="cuda", dtype=torch.float64 if prec == W.P64 else torch.float32)
    o = oracle.Oracle(grid, c["flow"])
    vol = torch.from_numpy(np.ascontiguousarray(1.0 / o.inner(o.J)).reshape(n)).to("cuda")
    out = torch.full((11,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        out.fill_(float("nan"))
        jz.jz_state_diagnostics_static(n, prec == W.P64, q_dev.data_ptr(), vol.data_ptr(), c["flow"]["gamma"],
                                       out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        r = out.cpu().numpy()
        scale = np.abs(Q.reshape(5, n)) @ (1.0 / o.inner(o.J).reshape(n))  # sum |Q_v| vol
        assert np.all(np.abs(r[0:5] - ref["sum"]) <= rtol * scale), (call, r[0:5], ref["sum"])
        for k, name in ((5, "rho_min"), (6, "rho_max"), (7, "p_min"), (8, "p_max"), (9, "mach_max")):
            assert r[k] == pytest.approx(ref[name], rel=1e-14), (call, name)
        assert r[10] == ref["nonfinite"] == 0
    g.close()


def test_static_scratch_rejects_oversize_input(jz):
    with pytest.raises(jz.JzError) as ei:
        jz.jz_state_diagnostics_static(2 ** 28 + 1, True, 256, 256, 1.4, 256, 0)
    assert ei.value.code == jz.JZ_EINVAL and "maximum" in str(ei.value)


def _numpy_reference(q64, vol, gamma, fp32):
    """Sums in FP64 and extrema, node by node, from the dense state."""
    ok = np.all(np.isfinite(q64), axis=0)
    qs = q64[:, ok].astype(np.float32 if fp32 else np.float64)
    T = qs.dtype.type
    ri = T(1) / qs[0]
    k = (qs[1] * qs[1] + qs[2] * qs[2] + qs[3] * qs[3]) * ri
    p = T(gamma - 1.0) * (qs[4] - T(0.5) * k)
    m2 = k / (T(gamma) * p)
    sums = (q64[:, ok] * vol[ok]).sum(axis=1)
    scale = (np.abs(q64[:, ok]) * vol[ok]).sum(axis=1)
    return sums, scale, q64[0, ok].min(), q64[0, ok].max(), p.min(), p.max(), float(np.sqrt(m2.max())), int((~ok).sum())


@pytest.mark.parametrize("fp64", [True, False])
def test_static_scratch_many_blocks_against_numpy(jz, fp64):
    """n = 3 * 65,536 + 17 nodes: three full reduction blocks and a partial
    fourth.  The global extrema sit in different blocks (one in the partial
    tail) and two nodes are non-finite, so the result is right only if every
    block's record reaches the ordered last-block combination.  Two calls in
    a row on one stream reuse the counter and records the first left."""
    import torch
    n = 3 * 65536 + 17
    rng = np.random.default_rng(11)
    rho = 1.0 + 0.2 * rng.uniform(-1, 1, n)
    u = rng.uniform(-1.5, 1.5, (3, n))
    p = (1.0 + 0.2 * rng.uniform(-1, 1, n)) / 1.4
    q = np.stack([rho, rho * u[0], rho * u[1], rho * u[2], p / 0.4 + 0.5 * rho * (u * u).sum(axis=0)])
    q[0, 70000] = 0.5            # density minimum in block 1
    q[0, n - 3] = 1.9            # density maximum in the partial block 3
    q[4, 140000] *= 3.0          # pressure maximum in block 2
    q[2, 5] = np.nan             # non-finite nodes in blocks 0 and 3
    q[4, n - 1] = np.inf
    if not fp64:
        q = q.astype(np.float32).astype(np.float64)  # exactly representable in FP32
    vol = rng.uniform(0.5, 2.0, n)
    sums, scale, rmin, rmax, pmin, pmax, mmax, nbad = _numpy_reference(q, vol, 1.4, not fp64)
    q_dev = torch.from_numpy(q).to(device="cuda", dtype=torch.float64 if fp64 else torch.float32)
    v_dev = torch.from_numpy(vol).to("cuda")
    out = torch.empty(11, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    prtol = 1e-14 if fp64 else 2e-6  # pressure / Mach in the state's type (FMA contraction on the GPU)
    for call in range(2):
        out.fill_(float("nan"))
        jz.jz_state_diagnostics_static(n, fp64, q_dev.data_ptr(), v_dev.data_ptr(), 1.4, out.data_ptr(),
                                       stream.cuda_stream)
        stream.synchronize()
        r = out.cpu().numpy()
        assert np.all(np.abs(r[0:5] - sums) <= 1e-13 * scale), (call, r[0:5], sums)
        assert r[5] == rmin == 0.5 and r[6] == rmax and r[6] == pytest.approx(1.9, rel=1e-7)
        assert r[7] == pytest.approx(pmin, rel=prtol) and r[8] == pytest.approx(pmax, rel=prtol)
        assert r[9] == pytest.approx(mmax, rel=prtol)
        assert r[10] == nbad == 2
