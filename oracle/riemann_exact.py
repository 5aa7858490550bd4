"""Exact solution of the Riemann problem for the 1D Euler equations of an ideal
gas (TEST INFRASTRUCTURE ONLY).

Method: the star-region pressure p* is the root of
    f(p) = f_L(p) + f_R(p) + (u_R - u_L) = 0,
where f_K is the velocity change across the left/right wave: a shock
(Rankine-Hugoniot) when p > p_K, a rarefaction (isentropic, Riemann
invariant) otherwise.  f is monotone and concave, so Newton's iteration from a
positive start converges.  This is the standard construction of Toro,
"Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4, written
here from those relations.  The solution is self-similar in x/t.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, ck, g):
    """Velocity jump across a K-wave and its derivative in p."""
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    e = (g - 1.0) / (2.0 * g)
    return 2.0 * ck / (g - 1.0) * ((p / pk) ** e - 1.0), 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


def star_state(left, right, gamma: float = 1.4, tol: float = 1e-15):
    """(p*, u*) of the Riemann problem with left/right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("initial data generate a vacuum")
    # two-rarefaction estimate as the starting point
    e = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** e + cr / pr ** e)) ** (1.0 / e)
    p = max(p, 1e-12)
    for _ in range(100):
        fl, dl = _fk(p, rl, pl, cl, g)
        fr, dr = _fk(p, rr, pr, cr, g)
        f = fl + fr + (ur - ul)
        pn = p - f / (dl + dr)
        pn = max(pn, 1e-14)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, xi, gamma: float = 1.4):
    """Exact (rho, u, p) at similarity coordinates xi = (x - x0) / t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    ps, us = star_state(left, right, g)
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for idx, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                if s <= sl:
                    r, v, q = rl, ul, pl
                else:
                    r, v, q = rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps
            else:  # left rarefaction
                csl = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                if s <= ul - cl:
                    r, v, q = rl, ul, pl
                elif s >= us - csl:
                    r, v, q = rl * (ps / pl) ** (1.0 / g), us, ps
                else:
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    v = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    r = rl * (c / cl) ** (2.0 / (g - 1.0))
                    q = pl * (c / cl) ** (2.0 * g / (g - 1.0))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                if s >= sr:
                    r, v, q = rr, ur, pr
                else:
                    r, v, q = rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps
            else:  # right rarefaction
                csr = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                if s >= ur + cr:
                    r, v, q = rr, ur, pr
                elif s <= us + csr:
                    r, v, q = rr * (ps / pr) ** (1.0 / g), us, ps
                else:
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    v = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    r = rr * (c / cr) ** (2.0 / (g - 1.0))
                    q = pr * (c / cr) ** (2.0 * g / (g - 1.0))
        rho[idx], u[idx], p[idx] = r, v, q
    return rho, u, p
