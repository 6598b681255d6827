"""Bounded device waits: a stage kernel whose data staging cannot complete
gives up, reports the failure and leaves the GPU usable.

The test switches on the grid's stall test (jz_set_stall_test): every TMA
copy of the stage kernels then expects 16 bytes that no copy delivers, so no
staging wait can succeed, and the waits give up after 2^16 cycles.  Nothing
traps or hangs: each kernel records the timeout, supplies the missing bytes
itself, lets its real copies land and returns.  jz_diagnostics must report
JZ_ETIMEOUT; after the flag is cleared and the state re-initialised, the
same grid must step bitwise like a grid that never stalled.  Both the FP32
vector-record kernel (the benchmark's) and the FP64 scalar kernel are
covered."""
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


@pytest.mark.parametrize("prec", [W.P32, W.P64])
def test_stalled_staging_reports_timeout_and_recovers(jz, prec):
    grid = W.jet_grid(40, 24, 20, map_amp=0.02, map_seed=1, precision=prec)
    flow = W.jet_flow()
    g = jz.Grid(grid).init(flow, 3)
    jz.jz_set_stall_test(g.h, True)
    g.nsteps(1, cfl=0.5)   # graph-captured step
    g.step(cfl=0.5)        # and a step launched directly
    with pytest.raises(jz.JzError) as ei:
        g.diagnostics(allow_nonfinite=True)
    assert ei.value.code == jz.JZ_ETIMEOUT
    assert "bounded device wait" in str(ei.value)

    jz.jz_set_stall_test(g.h, False)
    g.init(flow, 3)        # clears the sticky flag
    g.nsteps(3, cfl=0.5)
    got = g.download()
    d = g.diagnostics()
    g.close()
    ref_grid = jz.Grid(grid).init(flow, 3)
    ref_grid.nsteps(3, cfl=0.5)
    ref = ref_grid.download()
    dref = ref_grid.diagnostics()
    ref_grid.close()
    np.testing.assert_array_equal(got, ref)
    assert d["dt"] == dref["dt"] and d["nonfinite"] == 0


def test_stall_flag_is_checked(jz):
    g = jz.Grid(W.jet_grid(16, 12, 10, precision=W.P32)).init(W.jet_flow(), 0)
    with pytest.raises(jz.JzError) as ei:
        jz._check(jz.lib().jz_set_stall_test(g.h, 2))
    assert ei.value.code == jz.JZ_EINVAL
    g.close()
