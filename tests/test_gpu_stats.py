"""Time statistics of the axial velocity (the paper's <U>, u_rms, radial
profiles and potential core, Section 6) and restart files.

The running sums must equal a sequential loop over the sampled states
downloaded to the host (bitwise); the radial profile must equal the binning of
those statistics with the oracle's node coordinates; the potential-core length
of a state whose axial velocity falls linearly in x is known in closed form;
and a restarted run must continue bitwise as the uninterrupted one."""
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


@pytest.mark.parametrize("prec", [W.P64, W.P32])
def test_stats_equal_a_sequential_loop_over_samples(jz, prec):
    grid = W.jet_grid(48, 32, 24, map_amp=0.03, map_seed=1, precision=prec)
    g = jz.Grid(grid).init(W.jet_flow(), 3)
    st = jz.Stats(g)
    s = s2 = 0.0
    for _ in range(5):
        g.nsteps(1, cfl=0.5)
        st.sample()
        Q = g.download()
        u = Q[1] / Q[0]
        s = s + u
        s2 = s2 + u * u
    mean, rms = st.read()
    assert st.samples == 5
    m = s / 5
    np.testing.assert_array_equal(mean, m)
    np.testing.assert_array_equal(rms, np.sqrt(np.maximum(s2 / 5 - m * m, 0.0)))
    assert rms.max() > 0
    st.close()
    g.close()


def test_radial_profile_matches_binning_with_oracle_coordinates(jz):
    import oracle
    grid = W.jet_grid(31, 28, 28)  # unmapped: plane i sits at x = 30 i / 30
    flow = W.jet_flow()
    g = jz.Grid(grid).init(flow, 4)
    st = jz.Stats(g)
    for _ in range(3):
        g.nsteps(1, cfl=0.5)
        st.sample()
    mean, rms = st.read()
    nb, rmax = 6, 1.2
    pm, pr, pc = st.radial(5.0, nb, rmax)
    o = oracle.Oracle(grid, flow)
    y, z = o.inner(o.X[1])[:, :, 5], o.inner(o.X[2])[:, :, 5]
    r = np.sqrt(y * y + z * z)
    inside = r < rmax
    b = np.minimum(nb - 1, (r / rmax * nb).astype(int))
    for k in range(nb):
        sel = inside & (b == k)
        assert pc[k] == sel.sum()
        if sel.any():
            assert pm[k] == pytest.approx(mean[:, :, 5][sel].mean(), rel=1e-12)
            assert pr[k] == pytest.approx(rms[:, :, 5][sel].mean(), rel=1e-12, abs=1e-15)
    assert pc.sum() > 0 and pm[0] > 0.9 * flow["mach"]  # the jet core near the axis
    st.close()
    g.close()


def test_potential_core_length_of_a_linear_decay(jz):
    """u = M g(x), g = 1 for x <= 4, then falling linearly to 0.5 at x = 14:
    <U> drops below 0.95 M at x = 4 + 0.05 / 0.05 = 5."""
    grid = W.jet_grid(61, 12, 11)  # x_i = 0.5 i; odd nk: one axis line in k
    flow = W.jet_flow()
    M, gam = flow["mach"], flow["gamma"]
    g = jz.Grid(grid).init(flow, 0)
    x = 30.0 * np.arange(61) / 60.0
    gx = np.where(x <= 4.0, 1.0, np.maximum(0.5, 1.0 - 0.05 * (x - 4.0)))
    u = np.broadcast_to(M * gx, (11, 12, 61))
    Q = np.empty((5, 11, 12, 61))
    Q[0] = 1.0
    Q[1] = u
    Q[2] = Q[3] = 0.0
    Q[4] = 1.0 / (gam * (gam - 1.0)) + 0.5 * u * u
    g.upload(Q)
    st = jz.Stats(g)
    st.sample()
    assert st.core_length(M, 0.95) == pytest.approx(5.0, abs=1e-12)
    # at 0.4 M only the outflow face drops below (the far-field value there)
    assert 29.5 < st.core_length(M, 0.4) <= 30.0
    st.close()
    g.close()


@pytest.mark.parametrize("prec", [W.P64, W.P32])
def test_restart_continues_bitwise(jz, prec, tmp_path):
    grid = W.jet_grid(40, 24, 20, map_amp=0.03, map_seed=2, precision=prec)
    flow = W.jet_flow()
    a = jz.Grid(grid).init(flow, 6)
    a.nsteps(3, cfl=0.5)
    path = str(tmp_path / "restart.npz")
    a.save(path)
    a.nsteps(3, cfl=0.5)
    want, dwant = a.download(), a.diagnostics()
    b = jz.Grid(grid).init(flow, 0).load(path)
    b.nsteps(3, cfl=0.5)
    np.testing.assert_array_equal(b.download(), want)
    d = b.diagnostics()
    assert d["step"] == dwant["step"] == 6 and d["time"] == dwant["time"] and d["dt"] == dwant["dt"]
    a.close()
    b.close()


def test_cylinder_statistics(jz):
    """On the cylinder the axis is the centreline j = 0 (mean over its
    azimuths) and the radial profile bins each distinct node once: the
    closed-form core length of a linearly decaying axial velocity, and bin
    counts equal to the node count of each radius band."""
    ni, nj, nk = 61, 9, 13
    grid = W.cyl_grid(ni, nj, nk, length=30.0, radius=8.0, stretch_c=0.0)  # x_i = 0.5 i, r_j = j
    flow = W.jet_flow()
    M, gam = flow["mach"], flow["gamma"]
    g = jz.Grid(grid).init(flow, 0)
    x = 30.0 * np.arange(ni) / (ni - 1)
    gx = np.where(x <= 4.0, 1.0, np.maximum(0.5, 1.0 - 0.05 * (x - 4.0)))
    u = np.broadcast_to(M * gx, (nk, nj, ni))
    Q = np.empty((5, nk, nj, ni))
    Q[0] = 1.0
    Q[1] = u
    Q[2] = Q[3] = 0.0
    Q[4] = 1.0 / (gam * (gam - 1.0)) + 0.5 * u * u
    g.upload(Q)
    st = jz.Stats(g)
    st.sample()
    assert st.core_length(M, 0.95) == pytest.approx(5.0, abs=1e-12)
    nb, rmax = 5, 3.9  # r_j = j, bins 0.78 wide: j = 0, 1, 2, 3 in bins 0..3 (away from the edges), bin 4 empty
    pm, pr, pc = st.radial(5.0, nb, rmax)
    P = nk - 1
    np.testing.assert_array_equal(pc, [P, P, P, P, 0])
    np.testing.assert_allclose(pm[:4], 0.95 * M, rtol=1e-12)  # the plane x = 5, where u = 0.95 M
    st.close()
    g.close()
