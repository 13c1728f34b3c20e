"""Exact solution of the 1D Riemann problem for the ideal-gas Euler equations.

TEST INFRASTRUCTURE ONLY (pins for the shock-tube cases of Sec. 3.1: Sod, Lax,
Le Blanc are compared against the exact solution there).

Method: the standard textbook construction (Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", ch. 4): the star pressure solves
f_L(p) + f_R(p) + (u_R - u_L) = 0 with the shock (Rankine-Hugoniot) and
rarefaction (isentropic) branches of f_K; Newton iteration from the
two-rarefaction guess; the solution is then sampled along x/t.
"""
import math

import numpy as np


def _fK(p, rho, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        f = (p - pk) * s
        df = s * (1.0 - 0.5 * (p - pk) / (B + p))
    else:  # rarefaction
        pr = p / pk
        f = 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(WL, WR, gamma=1.4, tol=1e-15, itmax=200):
    """Return (p*, u*) for left/right primitive states (rho, u, p)."""
    rL, uL, pL = WL
    rR, uR, pR = WR
    g = gamma
    cL = math.sqrt(g * pL / rL)
    cR = math.sqrt(g * pR / rR)
    du = uR - uL
    if 2.0 / (g - 1.0) * (cL + cR) <= du:
        raise ValueError("vacuum is generated")
    z = (g - 1.0) / (2.0 * g)
    p = ((cL + cR - 0.5 * (g - 1.0) * du) / (cL / pL ** z + cR / pR ** z)) ** (1.0 / z)
    p = max(p, 1e-300)
    for _ in range(itmax):
        fL, dL = _fK(p, rL, pL, cL, g)
        fR, dR = _fK(p, rR, pR, cR, g)
        pn = p - (fL + fR + du) / (dL + dR)
        if pn <= 0.0:
            pn = 0.5 * p
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fK(p, rL, pL, cL, g)
    fR, _ = _fK(p, rR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def star_densities(WL, WR, gamma=1.4):
    p, u = star_state(WL, WR, gamma)
    g = gamma
    out = []
    for (r, _, pk) in (WL, WR):
        if p > pk:
            q = p / pk
            gr = (g - 1.0) / (g + 1.0)
            out.append(r * (q + gr) / (gr * q + 1.0))
        else:
            out.append(r * (p / pk) ** (1.0 / g))
    return p, u, out[0], out[1]


def sample(WL, WR, xi, gamma=1.4):
    """Primitive state (rho, u, p) at similarity coordinate xi = (x - x0)/t."""
    g = gamma
    rL, uL, pL = WL
    rR, uR, pR = WR
    p, u, rsL, rsR = star_densities(WL, WR, g)
    cL = math.sqrt(g * pL / rL)
    cR = math.sqrt(g * pR / rR)
    if xi <= u:  # left of the contact
        if p > pL:  # left shock
            SL = uL - cL * math.sqrt((g + 1.0) / (2.0 * g) * p / pL + (g - 1.0) / (2.0 * g))
            return (rL, uL, pL) if xi <= SL else (rsL, u, p)
        cs = cL * (p / pL) ** ((g - 1.0) / (2.0 * g))
        if xi <= uL - cL:
            return (rL, uL, pL)
        if xi >= u - cs:
            return (rsL, u, p)
        c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - xi))
        uu = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + xi)
        rr = rL * (c / cL) ** (2.0 / (g - 1.0))
        pp = pL * (c / cL) ** (2.0 * g / (g - 1.0))
        return (rr, uu, pp)
    if p > pR:  # right shock
        SR = uR + cR * math.sqrt((g + 1.0) / (2.0 * g) * p / pR + (g - 1.0) / (2.0 * g))
        return (rR, uR, pR) if xi >= SR else (rsR, u, p)
    cs = cR * (p / pR) ** ((g - 1.0) / (2.0 * g))
    if xi >= uR + cR:
        return (rR, uR, pR)
    if xi <= u + cs:
        return (rsR, u, p)
    c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - xi))
    uu = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + xi)
    rr = rR * (c / cR) ** (2.0 / (g - 1.0))
    pp = pR * (c / cR) ** (2.0 * g / (g - 1.0))
    return (rr, uu, pp)


def profile(WL, WR, x, x0, t, gamma=1.4):
    """Arrays rho, u, p at positions x and time t for a discontinuity at x0."""
    out = np.array([sample(WL, WR, (xx - x0) / t, gamma) for xx in np.asarray(x)])
    return out[:, 0], out[:, 1], out[:, 2]


def cell_average_profile(WL, WR, x_edges, x0, t, gamma=1.4, sub=64):
    """Cell averages of rho over cells [x_edges[i], x_edges[i+1]] (midpoint rule)."""
    x_edges = np.asarray(x_edges)
    out = []
    for a, b in zip(x_edges[:-1], x_edges[1:]):
        xs = a + (np.arange(sub) + 0.5) * (b - a) / sub
        r, _, _ = profile(WL, WR, xs, x0, t, gamma)
        out.append(r.mean())
    return np.array(out)
