"""Pins of the CPU FP64 oracle against facts that do not come from the oracle
itself: published generator outputs, closed forms, exact discrete identities,
textbook solutions and orders of accuracy.  Each test is chosen so that a
plausible slip somewhere in the oracle (a dropped term, a wrong sign, a
transposed index, a wrong coefficient) fails it.

Method: arXiv 2003.09926, Section 3 (filtered Navier-Stokes, Eqs. les,
q_mod, sutherland, tau_mod, vec-les, con-prop; centred differences with
Turkel-Vatsa dissipation; Jameson 5-stage Runge-Kutta; inflow and Riemann
far-field boundaries) and Section 4.3 (two-layer ghost fringe, five-point
dissipation stencil).
"""
import math
import os

import numpy as np
import pytest

from paper_2003_09926_gb300 import workloads as W

import states as ST

NG = 2
HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _set_all(o, Qin):
    """Interior state -> padded state with boundary conditions applied."""
    Q = o.new_state()
    Q[:, NG:-NG, NG:-NG, NG:-NG] = Qin
    o.apply_bc(Q)
    return Q


def _uniform(shape, rho, u, v, w, p):
    one = np.ones(shape)
    return ST.primitive_to_conserved(rho * one, u * one, v * one, w * one, p * one)


# ---------------------------------------------------------------------------
# counter-based generator
# ---------------------------------------------------------------------------

def test_splitmix64_published_vectors(orc):
    gamma = 0x9E3779B97F4A7C15
    for seed, idx, out in _golden("splitmix64.txt"):
        state = (int(seed) + int(idx) * gamma) & 0xFFFFFFFFFFFFFFFF
        assert orc.splitmix64(state) == int(out)


# ---------------------------------------------------------------------------
# metric terms (R6)
# ---------------------------------------------------------------------------

def test_metrics_affine_map_exact(orc):
    """x = A xi + b with a non-symmetric A: xi_k,x_m / J is the cofactor
    (det A) (A^-1)[k, m] and 1/J = det A, exactly (central differences of a
    linear map are exact).  A transposed operand or a wrong cyclic index
    fails this."""
    ni, nj, nk = 6, 5, 4
    d = W.periodic_grid(ni, nj, nk)
    A = np.array([[1.3, 0.2, -0.1], [0.15, 0.9, 0.3], [-0.25, 0.05, 1.1]])
    b = np.array([0.3, -0.2, 0.7])
    k, j, i = np.meshgrid(np.arange(-NG, nk + NG), np.arange(-NG, nj + NG), np.arange(-NG, ni + NG), indexing="ij")
    xi = np.stack([i, j, k]).astype(float)
    X = np.einsum("mk,k...->m...", A, xi) + b[:, None, None, None]
    o = orc.Oracle(d, W.jet_flow(), X=X)
    detA = np.linalg.det(A)
    cof = detA * np.linalg.inv(A)  # cof[k, m] = d xi_k / d x_m * det A
    S = o.inner(o.S).reshape(3, 3, -1)
    for kd in range(3):
        for m in range(3):
            np.testing.assert_allclose(S[kd, m], cof[kd, m], rtol=0, atol=1e-13)
    np.testing.assert_allclose(1.0 / o.inner(o.J), detA, rtol=1e-14)


def test_metrics_converge_to_analytic_derivatives(orc):
    """Unmapped stretched jet grid: the metrics reduce to products of
    coordinate derivatives (y_eta z_zeta etc., off-diagonals zero) and
    converge to the derivative of the coordinate map at second order."""
    errs = []
    for n in (129, 257, 513):
        d = W.jet_grid(3, n, n)
        o = orc.Oracle(d, W.jet_flow())
        S = o.inner(o.S).reshape(3, 3, o.desc["nk"], o.desc["nj"], o.desc["ni"])
        for a in range(3):
            for b in range(3):
                if a != b:
                    assert np.abs(S[a, b]).max() <= 1e-13
        # analytic d y / d eta from the coordinate map (fine 4th-order difference)
        e = 1e-3
        ys = np.array([(-o.base_coord(1, jj + 2 * e) + 8 * o.base_coord(1, jj + e) - 8 * o.base_coord(1, jj - e)
                        + o.base_coord(1, jj - 2 * e)) / (12 * e) for jj in range(n)])
        xs = 30.0 / 2
        # xi_x / J = y_eta z_zeta ; the z map equals the y map
        exact = ys[None, :, None] * ys[:, None, None] * np.ones((1, 1, 3))
        errs.append(np.abs(S[0, 0] - exact).max() / np.abs(exact).max())
        # 1/J = x_xi y_eta z_zeta
        jinv = 1.0 / o.inner(o.J)
        assert np.abs(jinv - xs * S[0, 0]).max() <= 1e-12 * np.abs(jinv).max()
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_metric_identity_on_mapped_grid(orc):
    """Conservative metric form: sum_k d_k (xi_k,x_m / J) = 0 at every node
    whose stencil is inside the grid, to roundoff (mapped, stretched grid)."""
    d = W.jet_grid(14, 12, 10, map_amp=0.3, map_seed=9)
    o = orc.Oracle(d, W.jet_flow())
    S = o.S.reshape(3, 3, *o.shape)
    for m in range(3):
        div = (0.5 * (S[0, m][:, :, 2:] - S[0, m][:, :, :-2]))[1:-1, 1:-1, :] \
            + (0.5 * (S[1, m][:, 2:, :] - S[1, m][:, :-2, :]))[1:-1, :, 1:-1] \
            + (0.5 * (S[2, m][2:, :, :] - S[2, m][:-2, :, :]))[:, 1:-1, 1:-1]
        inner = div[NG:-NG, NG:-NG, NG:-NG][1:-1, 1:-1, 1:-1]
        assert np.abs(inner).max() <= 1e-14 * np.abs(S).max()


# ---------------------------------------------------------------------------
# invariants of the full residual
# ---------------------------------------------------------------------------

def test_freestream_preservation_curved_grid(orc):
    """Uniform oblique Mach 1.4 flow on a strongly mapped periodic grid stays
    uniform: residual and 20-step drift at roundoff."""
    d = W.periodic_grid(12, 10, 8, hi=(2.0, 1.5, 1.2), map_amp=0.3, map_seed=5)
    o = orc.Oracle(d, W.jet_flow(re=1e3))
    sh = (8, 10, 12)
    Qin = _uniform(sh, 1.0, 1.4 * math.cos(0.3), 1.4 * math.sin(0.3), 0.2, 1.0 / 1.4)
    Q = _set_all(o, Qin)
    R = o.residual(Q)
    flux_scale = np.abs(o.S).max() * 1.4 ** 2
    assert np.abs(R).max() <= 1e-13 * flux_scale
    o.run(Q, 20, cfl=0.5)
    rel = np.abs(o.inner(Q) - Qin).max(axis=(1, 2, 3)) / np.abs(Qin).max(axis=(1, 2, 3))
    assert rel.max() <= 1e-13, rel


def test_discrete_conservation_periodic(orc):
    """Flux-difference form: sum over nodes of Q/J is constant to roundoff in
    a periodic mapped box, with inviscid, viscous, SGS and dissipation terms
    all active on a noisy field."""
    d = W.periodic_grid(12, 10, 8, hi=(2.0, 1.5, 1.2), map_amp=0.3, map_seed=5)
    o = orc.Oracle(d, W.jet_flow(re=2e3, cs=0.18))
    Q = _set_all(o, ST.random_state((8, 10, 12), seed=7))
    s0 = o.diagnostics(Q)["sum"]
    o.run(Q, 20, cfl=0.5)
    s1 = o.diagnostics(Q)["sum"]
    scale = np.array([abs(s0[0]), abs(s0[1]) + abs(s0[0]), abs(s0[2]) + abs(s0[0]), abs(s0[3]) + abs(s0[0]),
                      abs(s0[4])])
    assert (np.abs(s1 - s0) / scale).max() <= 1e-13
    assert np.abs(o.inner(Q) - o.inner(_set_all(o, ST.random_state((8, 10, 12), seed=7)))).max() > 1e-4


@pytest.mark.parametrize("k4", [0.0, 1.0 / 256.0, 1.0 / 32.0])
@pytest.mark.parametrize("mode", [1, 3, 7])
def test_rk_amplification_factor(orc, k4, mode):
    """Entropy wave (uniform u, p; density perturbation of 1e-6) on a uniform
    1-D periodic grid: the scheme is linear in the perturbation, so one step
    multiplies a Fourier mode by the stability polynomial of the 5-stage
    scheme, P(z) = 1 + z + z^2/2 + 3 z^3/16 + z^4/32 + z^5/128 (the products
    of alpha = 1/4, 1/6, 3/8, 1/2, 1), with
    z = -i dt U sin(theta)/h - dt J lambda~ 16 k4 sin^4(theta/2)
    (central difference symbol and fourth-difference dissipation symbol, with
    the anisotropic radius lambda~ = (U+c)(1 + 2 sqrt(c/(U+c))) / h^2 for
    sigma = 1/2 on a cube cell)."""
    N, eps, U = 32, 1e-6, 0.7
    h = 1.0 / N
    d = W.periodic_grid(N, 1, 1, hi=(1.0, h, h))
    o = orc.Oracle(d, W.jet_flow(re=0.0, cs=0.0, k4=k4, ic=W.IC_QUIESCENT))
    th = 2 * np.pi * mode / N
    rho = (1 + eps * np.cos(th * np.arange(N))).reshape(1, 1, N)
    one = np.ones((1, 1, N))
    Q = _set_all(o, ST.primitive_to_conserved(rho, U * one, 0 * one, 0 * one, one / 1.4))
    dt = 0.8 * h / (U + 1)
    r0 = np.fft.fft(o.inner(Q)[0, 0, 0] - 1)[mode]
    o.step(Q, dt=dt)
    r1 = np.fft.fft(o.inner(Q)[0, 0, 0] - 1)[mode]
    c = 1.0
    lam = (U + c) * (1 + 2 * np.sqrt(c / (U + c)))
    z = -1j * dt * U * np.sin(th) / h - dt / h * lam * 16 * k4 * np.sin(th / 2) ** 4
    P = 1 + z + z ** 2 / 2 + 3 * z ** 3 / 16 + z ** 4 / 32 + z ** 5 / 128
    assert abs(r1 / r0 - P) <= 1e-9


def _vortex(X, Y, t, L, u0, v0, beta=5.0, g=1.4):
    """Isentropic vortex (exact steady Euler solution advected by (u0, v0))
    in units rho_inf = 1, p_inf = 1/gamma: rho^(gamma-1) = 1 - (gamma-1)
    beta^2/(8 pi^2) exp(1 - r^2), p = rho^gamma / gamma, swirl (beta/2pi)
    exp((1-r^2)/2) (-dy, dx)."""
    dx = (X - u0 * t + L / 2) % L - L / 2
    dy = (Y - v0 * t + L / 2) % L - L / 2
    r2 = dx * dx + dy * dy
    A = (g - 1) * beta ** 2 / (8 * np.pi ** 2)
    rho = (1 - A * np.exp(1 - r2)) ** (1 / (g - 1))
    fac = beta / (2 * np.pi) * np.exp((1 - r2) / 2)
    return rho, u0 - fac * dy, v0 + fac * dx, 0 * rho, rho ** g / g


@pytest.mark.parametrize("mapped", [False, True])
def test_isentropic_vortex_second_order(orc, mapped):
    """Inviscid operator + RK on the isentropic vortex (periodic, 2-D, one
    node in z): L2 density error against the exact advected solution falls at
    order >= 1.8 (the scheme is second order in space and time)."""
    L, T = 12.0, 1.0
    errs = []
    for N in (32, 64, 128):
        h = L / N
        d = W.periodic_grid(N, N, 1, lo=(-6, -6, 0), hi=(6, 6, h), map_amp=0.1 if mapped else 0.0, map_seed=2)
        o = orc.Oracle(d, W.jet_flow(re=0.0, cs=0.0, ic=W.IC_QUIESCENT))
        X = o.inner(o.X)
        Q = _set_all(o, ST.primitive_to_conserved(*_vortex(X[0], X[1], 0.0, L, 0.5, 0.3)))
        n = int(np.ceil(T / (0.4 * h / 1.8)))
        o.run(Q, n, dt=T / n)
        rho_e = _vortex(X[0], X[1], T, L, 0.5, 0.3)[0]
        errs.append(np.sqrt(np.mean((o.inner(Q)[0] - rho_e) ** 2)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 1.8, (errs, orders)
    assert errs[-1] < 5e-4


def test_sod_shock_tube_converges(orc):
    """Pressure-sensor (k2) dissipation: two mirrored Sod problems on a
    periodic tube converge in L1 to the exact Riemann solution with no new
    density extrema (the textbook star state is checked first)."""
    import riemann_exact as RE
    ps, us, rl, rr = (float(v) for v in _golden("sod_star.txt")[0])
    got = RE.star_state((1, 0, 1), (0.125, 0, 0.1))
    np.testing.assert_allclose(got, (ps, us, rl, rr), rtol=2e-5)
    T, errs = 0.1, []
    for N in (100, 200, 400):
        h = 1.0 / N
        d = W.periodic_grid(N, 1, 1, hi=(1.0, h, h))
        o = orc.Oracle(d, W.jet_flow(re=0.0, cs=0.0, ic=W.IC_QUIESCENT))
        x = o.inner(o.X)[0, 0, 0]
        inside = (x >= 0.25) & (x < 0.75)
        rho = np.where(inside, 1.0, 0.125).reshape(1, 1, N)
        p = np.where(inside, 1.0, 0.1).reshape(1, 1, N)
        Q = _set_all(o, ST.primitive_to_conserved(rho, 0 * rho, 0 * rho, 0 * rho, p))
        n = int(np.ceil(T / (0.3 * h / 2.2)))
        o.run(Q, n, dt=T / n)
        xi = np.where(x < 0.5, (0.25 - x) / T, (x - 0.75) / T)
        rex = RE.sample((1, 0, 1), (0.125, 0, 0.1), xi)[0]
        r = o.inner(Q)[0, 0, 0]
        assert r.max() <= 1.0 + 1e-3 and r.min() >= 0.125 - 1e-3
        errs.append(np.mean(np.abs(r - rex)))
    assert errs[0] > errs[1] > errs[2] and errs[1] < 0.015, errs


def test_axis_permutation_equivariance(orc):
    """Relabelling the axes cyclically (x,y,z) -> (y,z,x) of grid, velocity
    and array permutes the residual the same way: catches any direction-
    dependent slip (metric, gradient, stress or dissipation index)."""
    n = 8
    d = W.periodic_grid(n, n, n, map_amp=0.25, map_seed=3)
    f = W.jet_flow(re=500.0, cs=0.18)
    o1 = orc.Oracle(d, f)
    Qin = ST.random_state((n, n, n), seed=11)
    Q1 = _set_all(o1, Qin)
    R1 = o1.residual(Q1)
    # new axis a' = old axis a+1:  new x-coord = old y-coord, array axes rolled
    def perm_field(F):  # (nk, nj, ni) arrays: new (k', j', i') = old (i, k, j)?
        return np.transpose(F, (2, 0, 1))
    X2 = np.stack([perm_field(o1.X[1]), perm_field(o1.X[2]), perm_field(o1.X[0])])
    o2 = orc.Oracle(d, f, X=X2)
    Qp = np.stack([perm_field(Qin[0]), perm_field(Qin[2]), perm_field(Qin[3]), perm_field(Qin[1]),
                   perm_field(Qin[4])])
    Q2 = _set_all(o2, Qp)
    R2 = o2.residual(Q2)
    R1p = np.stack([perm_field(R1[0]), perm_field(R1[2]), perm_field(R1[3]), perm_field(R1[1]), perm_field(R1[4])])
    scale = np.abs(R1).max(axis=(1, 2, 3))[[0, 2, 3, 1, 4]]
    err = np.abs(o2.inner(R2) - o2.inner(R1p)).max(axis=(1, 2, 3)) / scale
    assert err.max() <= 1e-12, err


# ---------------------------------------------------------------------------
# viscous flux and SGS: exact discrete results for polynomial fields
# ---------------------------------------------------------------------------

def _fill_padded(o, fn):
    """Evaluate a primitive-field function at every padded node (no BCs)."""
    X = o.X
    rho, u, v, w, p = fn(X[0], X[1], X[2])
    return np.ascontiguousarray(ST.primitive_to_conserved(rho, u, v, w, p))


def _viscous_part(orc, d, f, fn):
    """Viscous residual = R(mu) - R(mu=0) with dissipation off."""
    o = orc.Oracle(d, f)
    o0 = orc.Oracle(d, dict(f, re=0.0, cs=0.0))
    Q = _fill_padded(o, fn)
    return o, o.residual(Q) - o0.residual(Q)


def _interior(o, a):
    return o.inner(a)[..., 1:-1, 1:-1, 1:-1]


def test_viscous_momentum_quadratic_exact(orc):
    """Constant mu (T = 1), C_s = 0, quadratic velocity: node gradients and
    the centred difference of the (linear) stress are exact, so the viscous
    momentum residual is exactly -(1/J) [mu lap(u_i) + (mu/3) d_i div u], and
    the energy residual is the centred difference of the cubic u_i tau_ij:
    -(1/J) sum_j [d_j F_j + h_j^2/6 d_j^3 F_j]."""
    import sympy as sp
    hx, hy, hz = 0.1, 0.13, 0.07
    d = W.periodic_grid(7, 7, 7, hi=(6 * hx, 6 * hy, 6 * hz))
    d["bc"] = [W.BC_FARFIELD] * 6  # residual only, no periodic seam; node spacing (hi - lo) / (n - 1)
    f = W.jet_flow(re=50.0, cs=0.0, k2=0.0, k4=0.0)
    x, y, z = sp.symbols("x y z")
    rng = np.random.default_rng(5)
    coef = rng.uniform(-1, 1, size=(3, 10))
    mon = [sp.Integer(1), x, y, z, x * x, y * y, z * z, x * y, y * z, x * z]
    U = [sum(float(coef[c, m]) * mon[m] for m in range(10)) for c in range(3)]
    mu = f["mach"] / f["re"]
    Xs = (x, y, z)
    g = [[sp.diff(U[a], Xs[b]) for b in range(3)] for a in range(3)]
    div = g[0][0] + g[1][1] + g[2][2]
    tau = [[mu * (g[a][b] + g[b][a] - (sp.Rational(2, 3) * div if a == b else 0)) for b in range(3)] for a in range(3)]
    F5 = [sum(U[a] * tau[a][m] for a in range(3)) for m in range(3)]
    hs = (hx, hy, hz)
    mom = [sum(sp.diff(tau[a][m], Xs[m]) for m in range(3)) for a in range(3)]
    en = sum(sp.diff(F5[m], Xs[m]) + hs[m] ** 2 / 6 * sp.diff(F5[m], Xs[m], 3) for m in range(3))
    fu = [sp.lambdify((x, y, z), e, "numpy") for e in U]

    def fields(X, Y, Z):
        one = np.ones_like(X)
        return one, fu[0](X, Y, Z) * one, fu[1](X, Y, Z) * one, fu[2](X, Y, Z) * one, one / 1.4

    o, Rv = _viscous_part(orc, d, f, fields)
    Xi = _interior(o, o.X)
    vol = hx * hy * hz
    for a in range(3):
        exp = -vol * sp.lambdify((x, y, z), mom[a], "numpy")(Xi[0], Xi[1], Xi[2]) * np.ones_like(Xi[0])
        np.testing.assert_allclose(_interior(o, Rv)[1 + a], exp, rtol=1e-9, atol=1e-13)
    expE = -vol * sp.lambdify((x, y, z), en, "numpy")(Xi[0], Xi[1], Xi[2])
    np.testing.assert_allclose(_interior(o, Rv)[4], expE, rtol=1e-9, atol=1e-13)
    assert np.abs(_interior(o, Rv)[0]).max() == 0.0


def test_smagorinsky_pure_shear_exact(orc):
    """u = (a y^2/2 + b y, 0, 0), rho = 1, T = 1 on a cube grid (Delta = h):
    |S| = a y + b (> 0), mu_t = (C_s h)^2 |S|, tau_xy = (mu + mu_t)(a y + b)
    is quadratic in y, so the x-momentum residual is exactly
    -(1/J) [mu a + 2 (C_s h)^2 a (a y + b)]."""
    h, a, b = 0.1, 0.7, 2.0
    d = W.periodic_grid(7, 7, 7, hi=(0.6, 0.6, 0.6))
    d["bc"] = [W.BC_FARFIELD] * 6
    f = W.jet_flow(re=100.0, cs=0.18, k2=0.0, k4=0.0)

    def fields(X, Y, Z):
        one = np.ones_like(X)
        return one, a * Y * Y / 2 + b * Y, 0 * one, 0 * one, one / 1.4

    o, Rv = _viscous_part(orc, d, f, fields)
    mu = f["mach"] / f["re"]
    Y = _interior(o, o.X)[1]
    exp = -h ** 3 * (mu * a + 2 * (f["cs"] * h) ** 2 * a * (a * Y + b))
    np.testing.assert_allclose(_interior(o, Rv)[1], exp, rtol=1e-10)
    # Smagorinsky term is a sizeable part of the check
    assert np.abs(2 * (f["cs"] * h) ** 2 * a * (a * Y + b)).min() > 0.01 * mu * a


def test_vreman_vanishes_in_pure_shear(orc):
    """Vreman's model gives no eddy viscosity in pure shear: with
    u = (a y^2/2 + b y, 0, 0) only du/dy is non-zero, b_ij has one non-zero
    entry and all its 2x2 minors vanish, so the x-momentum residual is the
    laminar -(1/J) mu a (where Smagorinsky adds 2 (C_s h)^2 a (a y + b))."""
    h, a, b = 0.1, 0.7, 2.0
    d = W.periodic_grid(7, 7, 7, hi=(0.6, 0.6, 0.6))
    d["bc"] = [W.BC_FARFIELD] * 6
    f = W.jet_flow(re=100.0, cs=0.18, k2=0.0, k4=0.0, sgs=W.SGS_VREMAN)

    def fields(X, Y, Z):
        one = np.ones_like(X)
        return one, a * Y * Y / 2 + b * Y, 0 * one, 0 * one, one / 1.4

    o, Rv = _viscous_part(orc, d, f, fields)
    mu = f["mach"] / f["re"]
    got = _interior(o, Rv)[1]
    np.testing.assert_allclose(got, np.full(got.shape, -h ** 3 * mu * a), rtol=1e-12)


def test_vreman_linear_field_matches_invariant_form(orc):
    """u = A x (a general constant gradient g = A), rho = 1, T = 1, cube grid
    (Delta = h).  Vreman: nu_t = 2.5 C_s^2 h^2 sqrt(B / |A|^2), B the second
    invariant of M = A A^T, here taken as ((tr M)^2 - tr(M^2)) / 2 instead of
    the sum of principal minors.  The stress is constant, so the momentum
    residual vanishes and the energy residual is the exact centred difference
    of the linear u_a tau_am: -(1/J) (mu + nu_t) A_am (A_am + A_ma - 2/3 tr A delta_am)."""
    h = 0.1
    d = W.periodic_grid(7, 7, 7, hi=(0.6, 0.6, 0.6))
    d["bc"] = [W.BC_FARFIELD] * 6
    f = W.jet_flow(re=1000.0, cs=0.18, k2=0.0, k4=0.0, sgs=W.SGS_VREMAN)
    rng = np.random.default_rng(11)
    for trial in range(3):
        A = rng.uniform(-2, 2, size=(3, 3))

        def fields(X, Y, Z):
            one = np.ones_like(X)
            u = [A[c, 0] * X + A[c, 1] * Y + A[c, 2] * Z for c in range(3)]
            return one, u[0], u[1], u[2], one / 1.4

        o, Rv = _viscous_part(orc, d, f, fields)
        M = A @ A.T
        B = (np.trace(M) ** 2 - np.trace(M @ M)) / 2
        nut = 2.5 * f["cs"] ** 2 * h * h * np.sqrt(B / np.trace(M))
        mu = f["mach"] / f["re"]
        S = A + A.T - 2.0 / 3.0 * np.trace(A) * np.eye(3)
        expE = -h ** 3 * (mu + nut) * np.sum(A * S)
        got = _interior(o, Rv)[4]
        np.testing.assert_allclose(got, np.full(got.shape, expE), rtol=1e-11)
        for c in range(3):
            assert np.abs(_interior(o, Rv)[1 + c]).max() <= 1e-14
        assert nut > 0.2 * mu  # the eddy viscosity is a sizeable part of the check


def test_vreman_shear_plus_rotation_closed_form(orc):
    """u = (a y^2/2 + b y, c x, 0): s = a y + b and c are the only gradients,
    B = s^2 c^2, so nu_V(y) = 2.5 C_s^2 h^2 |c| s / sqrt(s^2 + c^2) (s > 0);
    tau_xy = (mu + nu_V)(s + c).  Node gradients are exact (quadratic u,
    linear v), so the x-momentum residual is -h^3 D_y[tau_xy], the
    y-momentum residual vanishes, and the energy residual is
    -h^3 [c tau_xy + D_y(u tau_xy)], D_y the centred difference."""
    h, a, b, c = 0.1, 0.9, 1.5, -2.0
    d = W.periodic_grid(7, 7, 7, hi=(0.6, 0.6, 0.6))
    d["bc"] = [W.BC_FARFIELD] * 6
    f = W.jet_flow(re=1000.0, cs=0.18, k2=0.0, k4=0.0, sgs=W.SGS_VREMAN)

    def fields(X, Y, Z):
        one = np.ones_like(X)
        return one, a * Y * Y / 2 + b * Y, c * X, 0 * one, one / 1.4

    o, Rv = _viscous_part(orc, d, f, fields)
    mu = f["mach"] / f["re"]
    Y = _interior(o, o.X)[1]

    def tau(y):
        s = a * y + b
        return (mu + 2.5 * f["cs"] ** 2 * h * h * abs(c) * s / np.sqrt(s * s + c * c)) * (s + c)

    def ut(y):
        return (a * y * y / 2 + b * y) * tau(y)

    D = lambda fn: (fn(Y + h) - fn(Y - h)) / (2 * h)
    np.testing.assert_allclose(_interior(o, Rv)[1], -h ** 3 * D(tau), rtol=1e-11)
    assert np.abs(_interior(o, Rv)[2]).max() <= 1e-15
    np.testing.assert_allclose(_interior(o, Rv)[4], -h ** 3 * (c * tau(Y) + D(ut)), rtol=1e-11)


def test_heat_flux_with_sgs_prandtl(orc):
    """T linear in x (rho = 1), u = (b y, 0, 0): grad T and |S| = b are exact,
    mu_e(x) = mu(T(x)) + (C_s h)^2 b, kappa_e = Cp (mu/Pr + mu_t/Pr_t).
    Energy residual: -(1/J) [D_x(kappa_e) T' + mu_e b^2]; y-momentum:
    -(1/J) D_x(mu_e) b, with D_x the centred difference (mu from the
    Sutherland law, itself pinned below)."""
    h, b, t1 = 0.1, 1.5, 0.4
    d = W.periodic_grid(7, 7, 7, lo=(0.2, 0, 0), hi=(0.8, 0.6, 0.6))
    d["bc"] = [W.BC_FARFIELD] * 6
    f = W.jet_flow(re=100.0, cs=0.18, k2=0.0, k4=0.0)
    g = f["gamma"]
    Cp = 1 / (g - 1)

    def fields(X, Y, Z):
        one = np.ones_like(X)
        T = 1.0 + t1 * X
        return one, b * Y, 0 * one, 0 * one, T / g

    o, Rv = _viscous_part(orc, d, f, fields)
    mut = (f["cs"] * h) ** 2 * b
    X = _interior(o, o.X)[0]
    mu = np.vectorize(o.sutherland)

    def kap(x):
        return Cp * (mu(1 + t1 * x) / f["pr"] + mut / f["prt"])

    def mue(x):
        return mu(1 + t1 * x) + mut

    D = lambda fn: (fn(X + h) - fn(X - h)) / (2 * h)
    np.testing.assert_allclose(_interior(o, Rv)[4], -h ** 3 * (D(kap) * t1 + mue(X) * b * b), rtol=1e-10)
    np.testing.assert_allclose(_interior(o, Rv)[2], -h ** 3 * D(mue) * b, rtol=1e-10)


def test_sutherland_law(orc):
    """mu(T_inf) = mu_inf = M/Re; with S1 = 110.4 K / 288.15 K the law maps
    the ISA sea-level viscosity to the tabulated 300 K value within 0.1%."""
    f = W.jet_flow()
    o = orc.Oracle(W.periodic_grid(4, 4, 4), f)
    assert o.mu_inf() == pytest.approx(1.4 / 1.57e6, rel=1e-15)
    assert o.sutherland(1.0) == pytest.approx(o.mu_inf(), rel=1e-15)
    (t0, mu0), (t1, mu1) = [(float(a), float(b)) for a, b in _golden("air_viscosity.txt")]
    assert mu0 * o.sutherland(t1 / t0) / o.sutherland(1.0) == pytest.approx(mu1, rel=1e-3)
    # high-temperature behaviour ~ T^(3/2)
    assert o.sutherland(400.0) / o.sutherland(100.0) == pytest.approx(8.0 * (100 + f["s1"]) / (400 + f["s1"]),
                                                                      rel=1e-13)


# ---------------------------------------------------------------------------
# boundary conditions, time step, initial state, diagnostics
# ---------------------------------------------------------------------------

def _prim(q, g=1.4):
    rho = q[0]
    u = q[1:4] / rho
    p = (g - 1) * (q[4] - 0.5 * rho * u @ u)
    return rho, u, p


def test_riemann_farfield_invariants(orc):
    """Subsonic far field: the outgoing invariant u_n + 2c/(g-1) is the
    interior one, the incoming u_n - 2c/(g-1) the freestream one; entropy
    p/rho^g and tangential velocity come from the upwind side.  Supersonic
    cases copy the upwind state; the freestream is a fixed point."""
    g = 1.4
    o = orc.Oracle(W.periodic_grid(4, 4, 4), W.jet_flow())
    rng = np.random.default_rng(3)
    for _ in range(50):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.3, 1.5) / g
        c = math.sqrt(g * p / rho)
        un = rng.uniform(-0.9, 0.9) * c
        ut = rng.normal(size=3)
        ut -= (ut @ n) * n
        u = ut + un * n
        qi = ST.primitive_to_conserved(rho, *u, p)
        qb = o.riemann(qi, n)
        rb, ub, pb = _prim(qb)
        cb = math.sqrt(g * pb / rb)
        assert ub @ n + 2 * cb / (g - 1) == pytest.approx(un + 2 * c / (g - 1), rel=1e-13)
        assert ub @ n - 2 * cb / (g - 1) == pytest.approx(-2.0 / (g - 1), rel=1e-13)
        if ub @ n > 0:
            assert pb / rb ** g == pytest.approx(p / rho ** g, rel=1e-12)
            np.testing.assert_allclose(ub - (ub @ n) * n, ut, atol=1e-13)
        else:
            assert pb / rb ** g == pytest.approx(1.0 / g, rel=1e-12)
            np.testing.assert_allclose(ub - (ub @ n) * n, 0.0, atol=1e-13)
    n = np.array([1.0, 0, 0])
    q_out = ST.primitive_to_conserved(1.0, 1.5, 0.2, 0.0, 1 / g)
    np.testing.assert_array_equal(o.riemann(q_out, n), q_out)
    q_in = ST.primitive_to_conserved(1.0, -1.5, 0.2, 0.0, 1 / g)
    np.testing.assert_allclose(o.riemann(q_in, n), ST.primitive_to_conserved(1.0, 0, 0, 0, 1 / g), rtol=1e-15)
    fs = ST.primitive_to_conserved(1.0, 0, 0, 0, 1 / g)
    np.testing.assert_allclose(o.riemann(fs, n), fs, rtol=1e-14, atol=1e-15)


def test_dt_uniform_grid_closed_form(orc):
    """Uniform Cartesian cells (hx, hy, hz), uniform state: the CFL step is
    cfl / [ sum_m (|u_m| + c)/h_m + 2 nu (1/hx^2 + 1/hy^2 + 1/hz^2) ],
    nu = max(4/3, gamma/Pr) mu / rho."""
    hx, hy, hz = 0.1, 0.05, 0.2
    d = W.periodic_grid(6, 6, 6, hi=(6 * hx, 6 * hy, 6 * hz))
    f = W.jet_flow(re=300.0)
    o = orc.Oracle(d, f)
    rho, u, v, w, p = 1.2, 0.5, -0.3, 0.2, 0.9 / 1.4
    Q = _set_all(o, _uniform((6, 6, 6), rho, u, v, w, p))
    c = math.sqrt(1.4 * p / rho)
    T = 1.4 * p / rho
    nu = max(4 / 3, 1.4 / 0.72) * o.sutherland(T) / rho
    rate = (abs(u) + c) / hx + (abs(v) + c) / hy + (abs(w) + c) / hz + 2 * nu * (1 / hx ** 2 + 1 / hy ** 2 + 1 / hz ** 2)
    assert o.step(Q, cfl=0.5) == pytest.approx(0.5 / rate, rel=1e-13)


def test_jet_initial_state_and_inflow(orc):
    """Jet state: rho = 1, p = 1/gamma, axial top-hat profile plus velocity
    noise of amplitude noise * M; the inflow plane is the noise-free
    profile, ghost layers copy the boundary node."""
    c = W.config0()
    o = orc.Oracle(c["grid"], c["flow"])
    Q = o.init(c["seed"])
    q = o.inner(Q)
    rho, p = q[0], 0.4 * (q[4] - 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / q[0])
    np.testing.assert_array_equal(rho[1:-1, 1:-1, 1:-1], 1.0)  # far-field nodes follow the Riemann BC
    np.testing.assert_array_equal(rho[:, :, 0], 1.0)
    X = o.inner(o.X)
    r = np.sqrt(X[1] ** 2 + X[2] ** 2)
    prof = np.vectorize(lambda rr: float(orc.lib().orc_jet_profile(orc.make_flow(c["flow"]), rr)))(r)
    # inflow plane (i = 0): exact profile, no noise
    np.testing.assert_allclose(q[1][:, :, 0], prof[:, :, 0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(q[2][:, :, 0], 0, atol=0)
    # interior: noise bounded by noise*M, roughly uniform
    noise = (q[1] - prof)[1:-1, 1:-1, 1:-1]
    amp = c["flow"]["noise"] * c["flow"]["mach"]
    assert np.abs(noise).max() <= amp and np.abs(noise).max() > 0.95 * amp
    assert abs(noise.mean()) < 0.05 * amp and abs(noise.std() / (amp / math.sqrt(3)) - 1) < 0.05
    np.testing.assert_allclose(p[1:-1, 1:-1, 1:-1], 1 / 1.4, rtol=1e-13)
    assert abs(prof.max() - 1.4) < 1e-3 and prof.min() < 1e-6
    # ghost layers copy the boundary node (zeroth order)
    np.testing.assert_array_equal(Q[:, :, :, 0], Q[:, :, :, 2])
    np.testing.assert_array_equal(Q[:, :, 1, :], Q[:, :, 2, :])
    np.testing.assert_array_equal(Q[:, -1, :, :], Q[:, -3, :, :])


def test_periodic_ghosts_wrap(orc):
    o = orc.Oracle(W.periodic_grid(5, 4, 3), W.jet_flow())
    Q = _set_all(o, ST.random_state((3, 4, 5), seed=2))
    np.testing.assert_array_equal(Q[..., 0], Q[..., 5])
    np.testing.assert_array_equal(Q[..., 1], Q[..., 6])
    np.testing.assert_array_equal(Q[..., 7], Q[..., 2])
    np.testing.assert_array_equal(Q[:, 0], Q[:, 3])
    np.testing.assert_array_equal(Q[:, :, -1], Q[:, :, 3])


def test_diagnostics_brute_force(orc):
    o = orc.Oracle(W.jet_grid(10, 8, 8, map_amp=0.1, map_seed=1), W.jet_flow())
    Q = o.init(5)
    dg = o.diagnostics(Q)
    q, J = o.inner(Q), o.inner(o.J)
    np.testing.assert_allclose(dg["sum"], (q / J).sum(axis=(1, 2, 3)), rtol=1e-13)
    assert dg["rho_min"] == q[0].min() and dg["nonfinite"] == 0
    Q[2, 5, 5, 5] = np.nan
    Q[4, 6, 5, 5] = np.inf
    assert o.diagnostics(Q)["nonfinite"] == 2


def test_jet_case_runs_and_stays_physical(orc):
    """Config-0 jet, 20 steps at CFL 0.5: finite, positive density and
    pressure, velocity bounded by the jet speed plus noise."""
    c = W.config0()
    o = orc.Oracle(c["grid"], c["flow"])
    Q = o.init(c["seed"])
    o.run(Q, c["steps"], cfl=c["cfl"])
    dg = o.diagnostics(Q)
    assert dg["nonfinite"] == 0 and dg["rho_min"] > 0.8 and dg["p_min"] > 0.5 / 1.4
    assert dg["mach_max"] < 1.6


# ---------------------------------------------------------------------------
# readings R5 (mapping), R7 (jet profile and noise) and R8 (edge tie-break),
# each evaluated by hand from its stated definition
# ---------------------------------------------------------------------------

_M64 = 0xFFFFFFFFFFFFFFFF


def _splitmix64(x: int) -> int:
    """SplitMix64 output for state x, written from the generator's published
    definition (the same vectors as tests/golden/splitmix64.txt pin it)."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def test_python_splitmix64_matches_published_vectors():
    gamma = 0x9E3779B97F4A7C15
    for seed, idx, out in _golden("splitmix64.txt"):
        assert _splitmix64((int(seed) + int(idx) * gamma) & _M64) == int(out)


def _unit53(r: int) -> float:
    return (r >> 11) / 9007199254740992.0


def test_jet_profile_hand_values(orc):
    """R7: u(r) = (M/2) (1 - tanh((r - 0.5) / (2 * 0.05))) with M = 1.4.  At
    r = 0.5 exactly M/2; one momentum thickness pair out (r = 0.6, 0.4)
    M/2 (1 -+ tanh 1).  A width of theta instead of 2 theta, a wrong radius
    or a wrong sign fails."""
    f = orc.make_flow(W.jet_flow())
    prof = lambda r: float(orc.lib().orc_jet_profile(f, r))  # noqa: E731
    M = 1.4
    assert prof(0.5) == 0.5 * M
    assert prof(0.6) == pytest.approx(0.5 * M * (1.0 - math.tanh(1.0)), rel=1e-14)
    assert prof(0.4) == pytest.approx(0.5 * M * (1.0 + math.tanh(1.0)), rel=1e-14)
    assert prof(0.0) == pytest.approx(0.5 * M * (1.0 + math.tanh(5.0)), rel=1e-15)
    assert prof(1.5) == pytest.approx(0.5 * M * (1.0 - math.tanh(10.0)), rel=1e-12)


def test_inflow_plane_is_the_hand_profile(orc):
    """The x = 0 plane of the config-0 jet holds rho = 1, p = 1/gamma,
    v = w = 0 and u = the R7 profile at r = sqrt(y^2 + z^2), with y and z
    from the R4 stretching formula evaluated here:
    y(s) = H G(s) / G(1), G(s) = s - (c/H)[tanh((H s - r_c)/w) + tanh((H s + r_c)/w)]."""
    c = W.config0()
    gd = c["grid"]
    o = orc.Oracle(gd, c["flow"])
    q = o.inner(o.init(c["seed"]))
    H, cc, w, rc = 8.0, gd["stretch_c"], gd["stretch_w"], gd["cluster_r"]

    def G(s):
        return s - (cc / H) * (math.tanh((H * s - rc) / w) + math.tanh((H * s + rc) / w))

    def coord(idx, n):
        return H * G(-1.0 + 2.0 * idx / (n - 1)) / G(1.0)

    M = c["flow"]["mach"]
    for k, j in ((0, 0), (5, 9), (16, 15), (31, 20), (13, 17)):
        y, z = coord(j, gd["nj"]), coord(k, gd["nk"])
        u = 0.5 * M * (1.0 - math.tanh((math.hypot(y, z) - 0.5) / 0.1))
        assert q[0, k, j, 0] == 1.0
        assert q[1, k, j, 0] == pytest.approx(u, rel=1e-13, abs=1e-15)
        assert q[2, k, j, 0] == 0.0 and q[3, k, j, 0] == 0.0
        assert q[4, k, j, 0] == pytest.approx(1.0 / (1.4 * 0.4) + 0.5 * u * u, rel=1e-14)


def test_initial_noise_hand_values(orc):
    """R7 noise: u_m += noise * M * (2 xi - 1), xi = top 53 bits of
    SplitMix64(seed XOR (3 lin + m)) / 2^53, lin = i + ni (j + nj k).  The
    transverse momenta of an interior node (rho = 1) are exactly that
    value; the axial one adds it to the profile.  A wrong linear index, a
    wrong stride 3 or a seed not XORed in fails."""
    gd = W.jet_grid(14, 10, 9)
    fl = W.jet_flow()
    o = orc.Oracle(gd, fl)
    seed = 0x5DEECE66D
    q = o.inner(o.init(seed))
    amp = fl["noise"] * fl["mach"]
    ni, nj = gd["ni"], gd["nj"]
    X = o.inner(o.X)
    for (i, j, k) in ((5, 7, 3), (1, 1, 1), (12, 8, 7), (7, 2, 5)):
        lin = i + ni * (j + nj * k)
        xi = [_unit53(_splitmix64(seed ^ (3 * lin + m))) for m in range(3)]
        r = math.hypot(X[1, k, j, i], X[2, k, j, i])
        prof = 0.5 * fl["mach"] * (1.0 - math.tanh((r - 0.5) / 0.1))
        assert q[0, k, j, i] == 1.0
        assert q[2, k, j, i] == amp * (2.0 * xi[1] - 1.0)
        assert q[3, k, j, i] == amp * (2.0 * xi[2] - 1.0)
        assert q[1, k, j, i] == pytest.approx(prof + amp * (2.0 * xi[0] - 1.0), rel=1e-15, abs=1e-16)


def test_mapping_offsets_hand_values(orc):
    """R5: x_d = base_d + a h_d prod_e sin(2 pi m_de idx_e / P_e + theta_de),
    m_de = 1 + SplitMix64(seed XOR 2c) mod 3 and theta_de = 2 pi * top-53
    bits of SplitMix64(seed XOR (2c + 1)), c = 3d + e; P_e = N_e - 1 (N_e in
    a periodic direction).  On an unstretched box the base coordinate and
    the spacing h_d are uniform, so every offset is evaluated here at
    interior, boundary and ghost indices.  A wrong wave-number draw, a
    wrong phase, N instead of N - 1 or a swapped (d, e) fails."""
    seed = 987654321
    gd = W.jet_grid(11, 9, 7, map_amp=0.05, map_seed=seed)
    gd["stretch_c"] = 0.0
    gd["bc"][4] = gd["bc"][5] = W.BC_PERIODIC  # z periodic: P = N
    o = orc.Oracle(gd, W.jet_flow())
    n = (gd["ni"], gd["nj"], gd["nk"])
    lo, hi = gd["lo"], gd["hi"]
    per = (False, False, True)
    P = [n[e] if per[e] else n[e] - 1 for e in range(3)]
    h = [(hi[d] - lo[d]) / P[d] for d in range(3)]
    m = [[1 + _splitmix64(seed ^ (2 * (3 * d + e))) % 3 for e in range(3)] for d in range(3)]
    th = [[2.0 * math.pi * _unit53(_splitmix64(seed ^ (2 * (3 * d + e) + 1))) for e in range(3)] for d in range(3)]
    mo, tho = o.map_params()
    np.testing.assert_array_equal(mo, np.array(m))
    np.testing.assert_array_equal(tho, np.array(th))
    for idx in ((3, 4, 2), (0, 0, 0), (10, 8, 6), (-2, 5, -1), (12, -1, 8), (7, 2, 4)):
        for d in range(3):
            base = lo[d] + h[d] * idx[d]
            prod = 1.0
            for e in range(3):
                prod *= math.sin(2.0 * math.pi * m[d][e] * idx[e] / P[e] + th[d][e])
            want = base + 0.05 * h[d] * prod
            got = o.X[d, idx[2] + NG, idx[1] + NG, idx[0] + NG]
            assert got == pytest.approx(want, rel=1e-13, abs=1e-13), (idx, d)


def test_boundary_edge_and_corner_tie_break(orc):
    """R8: on edges and corners the face latest in the order y-, y+, z-, z+,
    x+, x- sets the node.  A uniform state u = (2, 0.3, -2) (c = 1) makes
    every face's value distinct: x- is the inflow profile, x+ and z- see
    supersonic outflow (a copy of the adjacent interior node), z+ supersonic
    inflow (air at rest), y- and y+ subsonic Riemann states."""
    gd = W.jet_grid(8, 7, 6)
    gd["stretch_c"] = 0.0
    o = orc.Oracle(gd, W.jet_flow())
    ni, nj, nk = gd["ni"], gd["nj"], gd["nk"]
    g = 1.4
    Q = _set_all(o, _uniform((nk, nj, ni), 1.0, 2.0, 0.3, -2.0, 1.0 / g))
    q = o.inner(Q)
    rest = ST.primitive_to_conserved(1.0, 0.0, 0.0, 0.0, 1.0 / g)
    X = o.inner(o.X)

    def inflow(i, j, k):
        r = math.hypot(X[1, k, j, i], X[2, k, j, i])
        return ST.primitive_to_conserved(1.0, 0.5 * 1.4 * (1 - math.tanh((r - 0.5) / 0.1)), 0.0, 0.0, 1.0 / g)

    def interior(i, j, k):
        cl = lambda a, n: min(max(a, 1), n - 2)  # noqa: E731
        return q[:, cl(k, nk), cl(j, nj), cl(i, ni)]

    # the faces' own values, away from edges
    yface = q[:, 3, 0, 4]
    assert abs(yface[0] - 1.0) > 1e-3 and abs(q[0, 3, nj - 1, 4] - 1.0) > 1e-3
    np.testing.assert_array_equal(q[:, 0, 3, 4], interior(4, 3, 0))   # z-: copy
    np.testing.assert_allclose(q[:, nk - 1, 3, 4], rest, rtol=1e-15)   # z+: at rest
    cases = [  # (i, j, k) -> expected winner
        ((0, 0, 3), "x-"), ((0, nj - 1, 0), "x-"), ((0, 2, nk - 1), "x-"),
        ((ni - 1, 0, 3), "x+"), ((ni - 1, nj - 1, nk - 1), "x+"), ((ni - 1, 3, 0), "x+"),
        ((4, 0, 0), "z-"), ((4, nj - 1, 0), "z-"), ((4, 0, nk - 1), "z+"), ((4, nj - 1, nk - 1), "z+"),
    ]
    for (i, j, k), face in cases:
        got = q[:, k, j, i]
        if face == "x-":
            np.testing.assert_allclose(got, inflow(i, j, k), rtol=1e-14, atol=1e-15)
        elif face in ("x+", "z-"):
            np.testing.assert_array_equal(got, interior(i, j, k))
        else:
            np.testing.assert_allclose(got, rest, rtol=1e-15)
