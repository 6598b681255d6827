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
@pytest.mark.parametrize("prec,rtol", [(W.P64, 1e-12), (W.P32, 2.0 ** -22)])
def test_static_scratch_diagnostics_match_grid_diagnostics(jz, prec, rtol):
    import torch

    import oracle
    c = W.config0()
    grid = dict(c["grid"], map_amp=0.02, map_seed=1, precision=prec)
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
