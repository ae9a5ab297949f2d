"""Exact solution of the 1D Riemann problem for the Euler equations (ideal gas).

TEST INFRASTRUCTURE ONLY (a pin for the oracle's shock-tube results).

Written from the standard mathematics of the Riemann problem (e.g. Toro, "Riemann
Solvers and Numerical Methods for Fluid Dynamics", ch. 4): the star-region pressure p*
solves f_L(p*) + f_R(p*) + (u_R - u_L) = 0, with f_K the shock (Rankine-Hugoniot) or
rarefaction (isentropic) branch; the solution is then sampled along x/t.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _f(p, rho, pk, c, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)  # rarefaction


def star_state(left, right, g=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    F = lambda p: _f(p, rl, pl, cl, g) + _f(p, rr, pr, cr, g) + (ur - ul)
    pstar = brentq(F, 1e-12, 1e3 * max(pl, pr), xtol=1e-15, rtol=1e-15, maxiter=500)
    ustar = 0.5 * (ul + ur) + 0.5 * (_f(pstar, rr, pr, cr, g) - _f(pstar, rl, pl, cl, g))
    return pstar, ustar


def sample(left, right, xi, g=1.4):
    """(rho, u, p) at similarity coordinates xi = (x - x0)/t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi); u = np.empty_like(xi); p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for n, s in enumerate(xi.flat):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                rs = rl * ((ps / pl + gm) / (gm * ps / pl + 1.0))
                S = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                st = (rl, ul, pl) if s <= S else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / g)
                cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
                if s <= ul - cl:
                    st = (rl, ul, pl)
                elif s >= us - cs:
                    st = (rs, us, ps)
                else:
                    uu = 2.0 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    cc = 2.0 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    rr_ = rl * (cc / cl) ** (2.0 / (g - 1))
                    st = (rr_, uu, pl * (cc / cl) ** (2 * g / (g - 1)))
        else:
            if ps > pr:  # right shock
                rs = rr * ((ps / pr + gm) / (gm * ps / pr + 1.0))
                S = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                st = (rr, ur, pr) if s >= S else (rs, us, ps)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / g)
                cs = cr * (ps / pr) ** ((g - 1) / (2 * g))
                if s >= ur + cr:
                    st = (rr, ur, pr)
                elif s <= us + cs:
                    st = (rs, us, ps)
                else:
                    uu = 2.0 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    cc = 2.0 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    rr_ = rr * (cc / cr) ** (2.0 / (g - 1))
                    st = (rr_, uu, pr * (cc / cr) ** (2 * g / (g - 1)))
        rho.flat[n], u.flat[n], p.flat[n] = st
    return rho, u, p


def cell_average_density(left, right, x0, t, edges, g=1.4, sub=16):
    """Exact density averaged over cells with the given edges (sub-sampled midpoint rule)."""
    edges = np.asarray(edges)
    n = len(edges) - 1
    out = np.zeros(n)
    for k in range(sub):
        xs = edges[:-1] + (k + 0.5) / sub * (edges[1:] - edges[:-1])
        r, _, _ = sample(left, right, (xs - x0) / t, g)
        out += r
    return out / sub
