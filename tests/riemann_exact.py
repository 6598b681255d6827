"""Exact solution of the 1-D Riemann problem for the Euler equations of an
ideal gas (the classical two-wave pressure-function method: a Newton
iteration on p* for f_L(p) + f_R(p) + u_R - u_L = 0, then sampling of the
wave pattern along x/t).  Written for the tests; independent of the oracle."""
import math

import numpy as np


def _f(p, rho, pk, gamma):
    c = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    e = (gamma - 1.0) / (2.0 * gamma)
    return 2.0 * c / (gamma - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho * c)


def star_state(L, R, gamma=1.4):
    """(p*, u*, rho*_L, rho*_R) for left/right primitive states (rho, u, p)."""
    rl, ul, pl = L
    rr, ur, pr = R
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _f(p, rl, pl, gamma)
        fr, dr = _f(p, rr, pr, gamma)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p = max(1e-12, p - dp)
        if abs(dp) < 1e-15 * p:
            break
    fl, _ = _f(p, rl, pl, gamma)
    fr, _ = _f(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    g1 = (gamma - 1.0) / (gamma + 1.0)

    def rho_star(rk, pk):
        if p > pk:
            return rk * (p / pk + g1) / (g1 * p / pk + 1.0)
        return rk * (p / pk) ** (1.0 / gamma)

    return p, u, rho_star(rl, pl), rho_star(rr, pr)


def sample(L, R, xi, gamma=1.4):
    """Primitive state (rho, u, p) at similarity coordinate xi = x/t (arrays)."""
    rl, ul, pl = L
    rr, ur, pr = R
    ps, us, rsl, rsr = star_state(L, R, gamma)
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    xi = np.asarray(xi, dtype=float)
    rho, u, p = np.empty_like(xi), np.empty_like(xi), np.empty_like(xi)
    for n, s in np.ndenumerate(xi):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
                st = (rl, ul, pl) if s < sl else (rsl, us, ps)
            else:  # left rarefaction
                csl = cl * (ps / pl) ** ((gamma - 1) / (2 * gamma))
                if s < ul - cl:
                    st = (rl, ul, pl)
                elif s > us - csl:
                    st = (rsl, us, ps)
                else:
                    uu = 2 / (gamma + 1) * (cl + (gamma - 1) / 2 * ul + s)
                    cc = 2 / (gamma + 1) * (cl + (gamma - 1) / 2 * (ul - s))
                    rr_ = rl * (cc / cl) ** (2 / (gamma - 1))
                    st = (rr_, uu, pl * (cc / cl) ** (2 * gamma / (gamma - 1)))
        else:
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
                st = (rr, ur, pr) if s > sr else (rsr, us, ps)
            else:  # right rarefaction
                csr = cr * (ps / pr) ** ((gamma - 1) / (2 * gamma))
                if s > ur + cr:
                    st = (rr, ur, pr)
                elif s < us + csr:
                    st = (rsr, us, ps)
                else:
                    uu = 2 / (gamma + 1) * (-cr + (gamma - 1) / 2 * ur + s)
                    cc = 2 / (gamma + 1) * (cr - (gamma - 1) / 2 * (ur - s))
                    rr_ = rr * (cc / cr) ** (2 / (gamma - 1))
                    st = (rr_, uu, pr * (cc / cr) ** (2 * gamma / (gamma - 1)))
        rho[n], u[n], p[n] = st
    return rho, u, p
