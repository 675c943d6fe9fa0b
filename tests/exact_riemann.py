"""Exact solution of the 1D Riemann problem for the ideal-gas Euler equations.

Written from the textbook derivation (Toro, "Riemann Solvers and Numerical
Methods for Fluid Dynamics", ch. 4): the star-region pressure is the root of
f(p) = f_L(p) + f_R(p) + (u_R - u_L), where f_K is the shock (Rankine-Hugoniot)
branch for p > p_K and the rarefaction (isentropic) branch otherwise; the
solution is then sampled on the similarity variable x/t.  Used only as an
independent pin of the oracle (shock-tube convergence test).
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    r = (p / pk) ** ((g - 1.0) / (2.0 * g))
    f = 2.0 * ck / (g - 1.0) * (r - 1.0)
    df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rhoL, uL, pL, rhoR, uR, pR, g):
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    p = max(1e-12, 0.5 * (pL + pR))
    for _ in range(200):
        fL, dL = _fk(p, rhoL, pL, cL, g)
        fR, dR = _fk(p, rhoR, pR, cR, g)
        f = fL + fR + (uR - uL)
        pn = p - f / (dL + dR)
        if pn <= 0:
            pn = 0.5 * p
        if abs(pn - p) <= 1e-14 * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fk(p, rhoL, pL, cL, g)
    fR, _ = _fk(p, rhoR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def sample(xi, left, right, g):
    """Exact (rho, u, p) at similarity coordinate xi = (x - x0)/t."""
    rhoL, uL, pL = left
    rhoR, uR, pR = right
    ps, us = star_state(rhoL, uL, pL, rhoR, uR, pR, g)
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    gm = (g - 1.0) / (g + 1.0)
    if xi <= us:  # left of contact
        if ps > pL:  # left shock
            rs = rhoL * (ps / pL + gm) / (gm * ps / pL + 1.0)
            S = uL - cL * math.sqrt((g + 1.0) / (2 * g) * ps / pL + (g - 1.0) / (2 * g))
            return (rhoL, uL, pL) if xi <= S else (rs, us, ps)
        rs = rhoL * (ps / pL) ** (1.0 / g)
        cs = cL * (ps / pL) ** ((g - 1.0) / (2 * g))
        head, tail = uL - cL, us - cs
        if xi <= head:
            return rhoL, uL, pL
        if xi >= tail:
            return rs, us, ps
        u = 2.0 / (g + 1.0) * (cL + (g - 1.0) / 2.0 * uL + xi)
        c = 2.0 / (g + 1.0) * (cL + (g - 1.0) / 2.0 * (uL - xi))
        rho = rhoL * (c / cL) ** (2.0 / (g - 1.0))
        p = pL * (c / cL) ** (2.0 * g / (g - 1.0))
        return rho, u, p
    if ps > pR:  # right shock
        rs = rhoR * (ps / pR + gm) / (gm * ps / pR + 1.0)
        S = uR + cR * math.sqrt((g + 1.0) / (2 * g) * ps / pR + (g - 1.0) / (2 * g))
        return (rhoR, uR, pR) if xi >= S else (rs, us, ps)
    rs = rhoR * (ps / pR) ** (1.0 / g)
    cs = cR * (ps / pR) ** ((g - 1.0) / (2 * g))
    head, tail = uR + cR, us + cs
    if xi >= head:
        return rhoR, uR, pR
    if xi <= tail:
        return rs, us, ps
    u = 2.0 / (g + 1.0) * (-cR + (g - 1.0) / 2.0 * uR + xi)
    c = 2.0 / (g + 1.0) * (cR - (g - 1.0) / 2.0 * (uR - xi))
    rho = rhoR * (c / cR) ** (2.0 / (g - 1.0))
    p = pR * (c / cR) ** (2.0 * g / (g - 1.0))
    return rho, u, p


def cell_average_density(xc, dx, t, x0, left, right, g, sub=16):
    """Cell averages of the exact density (midpoint rule on `sub` points)."""
    out = np.empty(xc.size)
    offs = (np.arange(sub) + 0.5) / sub - 0.5
    for i, x in enumerate(xc):
        out[i] = np.mean([sample((x + o * dx - x0) / t, left, right, g)[0] for o in offs])
    return out
