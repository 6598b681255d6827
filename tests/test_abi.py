"""C-ABI library checks that need no GPU: it loads, exports every function
include/jz.h declares, sizes buffers by plain arithmetic and rejects bad
descriptors with JZ_EINVAL before touching CUDA."""
import ctypes as C

import pytest

from paper_2003_09926_gb300 import jz
from paper_2003_09926_gb300 import workloads as W


@pytest.fixture(scope="module")
def L():
    from paper_2003_09926_gb300 import build
    build.build()
    return jz.lib()


def test_exports_every_header_function(L):
    names = jz.header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/jz.h but not exported"


def test_grid_bytes_layout(L):
    for prec, es, ms in ((W.P64, 8, 8), (W.P32_M64, 4, 8), (W.P32, 4, 4)):
        d = W.jet_grid(48, 32, 32, precision=prec)
        nb = jz.jz_grid_bytes(d)
        pitch = (48 + 4 + 31) // 32 * 32
        npad = pitch * 36 * 36
        assert nb >= 3 * 5 * npad * es + 10 * npad * ms
        assert nb <= 3 * 5 * npad * es + 10 * npad * ms + 256 * 1024 + 32 * 32 * 8


def test_paper_scale_footprint(L):
    """1024 x 1024 x 960 FP32 grid: three FP32 states and FP32 metrics,
    about 100 B per point plus padding -- fits one GB300."""
    nb = jz.jz_grid_bytes(W.config2()["grid"])
    pts = 1024 * 1024 * 960
    assert 100 * pts <= nb <= 1.12 * 100 * pts
    assert nb < 150e9


@pytest.mark.parametrize("mutate,msg", [
    (lambda d: d.update(ni=2), "too few"),
    (lambda d: d.update(precision=7), "precision"),
    (lambda d: d.update(bc=[0, 2, 2, 2, 2, 2]), "periodic"),
    (lambda d: d.update(bc=[9, 2, 2, 2, 2, 2]), "boundary kind"),
    (lambda d: d.update(hi=[0.0, 8.0, 8.0]), "extent"),
    (lambda d: d.update(ni=64, nj=1 << 15, nk=1 << 15), "too large"),  # 2^31 rows of 32 nodes
])
def test_bad_descriptors_rejected(L, mutate, msg):
    d = W.jet_grid(16, 16, 16)
    mutate(d)
    with pytest.raises(jz.JzError) as ei:
        jz.jz_grid_bytes(d)
    assert ei.value.code == jz.JZ_EINVAL
    assert msg in str(ei.value)


def test_create_rejects_bad_buffers_without_cuda(L):
    d = jz.make_desc(W.jet_grid(16, 16, 16))
    h = C.c_void_p()
    assert L.jz_grid_create(C.byref(d), None, 1 << 30, None, C.byref(h)) == jz.JZ_EINVAL
    assert L.jz_grid_create(C.byref(d), C.c_void_p(0x1000 + 8), 1 << 30, None, C.byref(h)) == jz.JZ_EINVAL
    assert "aligned" in jz.last_error()
    assert L.jz_grid_create(C.byref(d), C.c_void_p(0x100000), 1024, None, C.byref(h)) == jz.JZ_ENOMEM


def test_null_handles_rejected(L):
    assert L.jz_rk_step(None, 0.5, 0.0) == jz.JZ_EINVAL
    assert L.jz_grid_destroy(None) == jz.JZ_OK
    assert L.jz_set_step_diagnostics(None, 1) == jz.JZ_EINVAL
    assert L.jz_step_diagnostics_async(None, None) == jz.JZ_EINVAL
    assert L.jz_diagnostics_async(None, None) == jz.JZ_EINVAL
    n = C.c_uint64()
    assert L.jz_launch_count(C.byref(n)) == jz.JZ_OK


@pytest.mark.parametrize("mutate,msg", [
    (lambda d: d.update(nk=14), "nk - 1 even"),
    (lambda d: d.update(map_amp=0.01), "mapping"),
    (lambda d: d.update(lo=[0.0, 0.5, 0.0]), "lo[1] = 0"),
    (lambda d: d.update(bc=[W.BC_INFLOW, W.BC_FARFIELD, W.BC_FARFIELD, W.BC_FARFIELD, W.BC_PERIODIC,
                            W.BC_PERIODIC]), "JZ_BC_AXIS"),
    (lambda d: d.update(bc=[W.BC_INFLOW, W.BC_FARFIELD, W.BC_AXIS, W.BC_FARFIELD, W.BC_FARFIELD,
                            W.BC_FARFIELD]), "periodic in k"),
    (lambda d: d.update(geom=W.GEOM_BOX), "centreline"),
    (lambda d: d.update(geom=5), "geometry"),
])
def test_bad_cylinder_descriptors_rejected(L, mutate, msg):
    d = W.cyl_grid(16, 8, 13)
    assert jz.jz_grid_bytes(d) > 0
    mutate(d)
    with pytest.raises(jz.JzError) as ei:
        jz.jz_grid_bytes(d)
    assert ei.value.code == jz.JZ_EINVAL
    assert msg in str(ei.value)


def test_cylinder_blocks_split_in_i_only(L):
    d = W.cyl_grid(40, 8, 13)
    assert jz.jz_block_bytes(d, (0, 0, 0), (19, 7, 12)) > 0
    for o0, o1 in (((0, 0, 0), (39, 3, 12)), ((0, 0, 0), (39, 7, 5))):
        with pytest.raises(jz.JzError) as ei:
            jz.jz_block_bytes(d, o0, o1)
        assert ei.value.code == jz.JZ_EINVAL


def test_serving_selection_is_oldest_first_until_filled():
    from paper_2003_09926_gb300 import serve
    reqs = [serve.Request(i, W.jet_grid(10 + i, 10, 10), W.jet_flow(), 0, 5, arrival=a)
            for i, a in enumerate([0.3, 0.1, 0.2, 0.0])]
    resident = [dict(req=r) for r in reqs]
    pts = {r.rid: serve.updated_points(r.grid) for r in reqs}
    assert serve.select_cases(resident, None) == resident
    one = serve.select_cases(resident, 1)
    assert [c["req"].rid for c in one] == [3]
    two = serve.select_cases(resident, pts[3] + 1)
    assert [c["req"].rid for c in two] == [3, 1]
    assert [c["req"].rid for c in serve.select_cases(resident, 10**9)] == [3, 1, 2, 0]



def test_largest_row_count_accepted(L):
    """Just below the 32-bit row limit the descriptor is valid (sizing only)."""
    d = dict(W.jet_grid(16, 16, 16), ni=32, nj=1 << 15, nk=1 << 15)
    assert jz.jz_grid_bytes(d) > 0
