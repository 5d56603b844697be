"""Exact solution of the Riemann problem for the 1-D Euler equations of an ideal gas.

Written from the textbook construction (E. F. Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", ch. 4): the star-region pressure is the
root of f_L(p) + f_R(p) + (u_R - u_L) = 0, with f_K the shock (Rankine-Hugoniot)
or rarefaction (isentropic, Riemann-invariant) branch; the solution is then
sampled on rays x/t.  Used only as a closed-form pin for the B = 0 shock tube.
"""
from __future__ import annotations

import math

import numpy as np


def _fK(p, rho, pK, cK, g):
    if p > pK:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        s = math.sqrt(A / (p + B))
        f = (p - pK) * s
        df = s * (1.0 - 0.5 * (p - pK) / (B + p))
    else:       # rarefaction
        f = 2.0 * cK / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = (1.0 / (rho * cK)) * (p / pK) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(WL, WR, g):
    """(p*, u*) for left/right primitive states W = (rho, u, p)."""
    rl, ul, pl = WL
    rr, ur, pr = WR
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(100):
        fl, dfl = _fK(p, rl, pl, cl, g)
        fr, dfr = _fK(p, rr, pr, cr, g)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-14)
        if abs(pn - p) / (0.5 * (pn + p)) < 1e-15:
            p = pn
            break
        p = pn
    fl, _ = _fK(p, rl, pl, cl, g)
    fr, _ = _fK(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(WL, WR, g, xi):
    """Primitive (rho, u, p) on rays xi = x/t (array)."""
    rl, ul, pl = WL
    rr, ur, pr = WR
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    ps, us = star_state(WL, WR, g)
    gm = (g - 1.0) / (g + 1.0)
    xi = np.asarray(xi, dtype=np.float64)
    out = np.zeros((3,) + xi.shape)
    for idx, S in np.ndenumerate(xi):
        if S <= us:  # left of the contact
            if ps > pl:
                SL = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if S <= SL:
                    W = (rl, ul, pl)
                else:
                    W = (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)
            else:
                SHL = ul - cl
                cml = cl * (ps / pl) ** ((g - 1) / (2 * g))
                STL = us - cml
                if S <= SHL:
                    W = (rl, ul, pl)
                elif S >= STL:
                    W = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    base = 2.0 / (g + 1) + (g - 1) / ((g + 1) * cl) * (ul - S)
                    W = (rl * base ** (2.0 / (g - 1)), 2.0 / (g + 1) * (cl + 0.5 * (g - 1) * ul + S),
                         pl * base ** (2.0 * g / (g - 1)))
        else:        # right of the contact
            if ps > pr:
                SR = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if S >= SR:
                    W = (rr, ur, pr)
                else:
                    W = (rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps)
            else:
                SHR = ur + cr
                cmr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                STR = us + cmr
                if S >= SHR:
                    W = (rr, ur, pr)
                elif S <= STR:
                    W = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    base = 2.0 / (g + 1) - (g - 1) / ((g + 1) * cr) * (ur - S)
                    W = (rr * base ** (2.0 / (g - 1)), 2.0 / (g + 1) * (-cr + 0.5 * (g - 1) * ur + S),
                         pr * base ** (2.0 * g / (g - 1)))
        out[(slice(None),) + idx] = W
    return out


def shock_speed(WL, WR, g):
    """Speed of the right-moving shock (requires p* > p_R)."""
    rr, ur, pr = WR
    cr = math.sqrt(g * pr / rr)
    ps, _ = star_state(WL, WR, g)
    return ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
