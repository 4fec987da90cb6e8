"""Exact solution of the 1D Euler Riemann problem (ideal gas), a test helper.

The star pressure p* solves f_L(p) + f_R(p) + (v_R - v_L) = 0, where f_K is
the velocity jump across a shock (p > p_K, Rankine-Hugoniot) or a rarefaction
(p <= p_K, isentropic) connecting state K to pressure p; f is increasing in
p, so p* is bracketed and found by Brent's method.  The solution is then
sampled at x/t (the classical exact solver of gas dynamics textbooks, written
here from those relations).  Used only to measure errors of computed
solutions; it holds none of the method's arithmetic.
"""
import math

import numpy as np
from scipy.optimize import brentq


def _f(p, rho, pk, g):
    c = math.sqrt(g * pk / rho)
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def vacuum(left, right, g=1.4):
    (rl, vl, pl), (rr, vr, pr) = left, right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    return 2.0 * (cl + cr) / (g - 1.0) <= vr - vl


def star(left, right, g=1.4):
    """(p*, v*) of the Riemann problem with primitive states (rho, v, p)."""
    (rl, vl, pl), (rr, vr, pr) = left, right
    if vacuum(left, right, g):
        raise ValueError("the data generate vacuum")
    F = lambda p: _f(p, rl, pl, g) + _f(p, rr, pr, g) + (vr - vl)
    lo, hi = 1e-14 * min(pl, pr), max(pl, pr)
    while F(hi) < 0.0:
        hi *= 4.0
    ps = brentq(F, lo, hi, xtol=1e-15 * hi, rtol=1e-15, maxiter=500)
    vs = 0.5 * (vl + vr) + 0.5 * (_f(ps, rr, pr, g) - _f(ps, rl, pl, g))
    return ps, vs


def max_speed(left, right, g=1.4):
    """Largest |wave speed| of the solution."""
    (rl, vl, pl), (rr, vr, pr) = left, right
    ps, vs = star(left, right, g)
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    sL = vl - cl * (math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g)) if ps > pl else 1.0)
    sR = vr + cr * (math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g)) if ps > pr else 1.0)
    return max(abs(sL), abs(sR), abs(vs))


def sample(left, right, s, g=1.4):
    """Primitive (rho, v, p) arrays at the similarity coordinates s = (x - x0)/t."""
    (rl, vl, pl), (rr, vr, pr) = left, right
    ps, vs = star(left, right, g)
    s = np.asarray(s, dtype=np.float64)
    out = np.empty((3,) + s.shape)
    gm, gp = g - 1.0, g + 1.0
    for idx, si in np.ndenumerate(s):
        if si <= vs:   # left of the contact
            rho, v, p, sgn = rl, vl, pl, 1.0
        else:
            rho, v, p, sgn = rr, vr, pr, -1.0
        c = math.sqrt(g * p / rho)
        # mirror the right side onto the left-side formulas: x -> -x, v -> -v
        vv, ss, vst = sgn * v, sgn * si, sgn * vs
        if ps > p:     # shock
            S = vv - c * math.sqrt(gp / (2 * g) * ps / p + gm / (2 * g))
            if ss <= S:
                r, u, q = rho, vv, p
            else:
                r = rho * (ps / p + gm / gp) / (gm / gp * ps / p + 1.0)
                u, q = vst, ps
        else:          # rarefaction
            head = vv - c
            cs = c * (ps / p) ** (gm / (2 * g))
            tail = vst - cs
            if ss <= head:
                r, u, q = rho, vv, p
            elif ss >= tail:
                r, u, q = rho * (ps / p) ** (1.0 / g), vst, ps
            else:
                cf = 2.0 / gp * (c + gm / 2.0 * (vv - ss))
                u = 2.0 / gp * (c + gm / 2.0 * vv + ss)
                r = rho * (cf / c) ** (2.0 / gm)
                q = p * (cf / c) ** (2.0 * g / gm)
        out[0][idx], out[1][idx], out[2][idx] = r, sgn * u, q
    return out
