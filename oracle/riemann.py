"""Exact solution of the one-dimensional Riemann problem for an ideal gas.

TEST INFRASTRUCTURE (part of the oracle).  The closed-form Sod shock tube
solution that the SPH oracle and the CUDA path are checked against.  This is
the textbook construction (two nonlinear waves separated by a contact; the star
pressure is the root of the pressure function, found by Newton iteration; the
solution is self-similar in x/t), written from the gas dynamics, not from any
listing.

Pinned by ``tests/test_oracle_sod.py`` against the textbook star state of the
standard Sod problem (p* = 0.30313, u* = 0.92745 for rho_L = 1, p_L = 1,
rho_R = 0.125, p_R = 0.1, gamma = 1.4).
"""
from __future__ import annotations

import math

import numpy as np


def _wave_fn(p, rho, pk, g):
    """Velocity change across a wave from state (rho, pk) to pressure p, and its derivative."""
    a = math.sqrt(g * pk / rho)
    if p > pk:  # shock: Rankine-Hugoniot
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction: isentropic
    e = (g - 1.0) / (2.0 * g)
    return (2.0 * a / (g - 1.0)) * ((p / pk) ** e - 1.0), (1.0 / (rho * a)) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


def star_state(rhoL, uL, pL, rhoR, uR, pR, g):
    """Pressure and velocity between the two nonlinear waves."""
    p = max(1e-12, 0.5 * (pL + pR))
    for _ in range(100):
        fL, dL = _wave_fn(p, rhoL, pL, g)
        fR, dR = _wave_fn(p, rhoR, pR, g)
        f = fL + fR + (uR - uL)
        pn = p - f / (dL + dR)
        pn = max(pn, 1e-12)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _wave_fn(p, rhoL, pL, g)
    fR, _ = _wave_fn(p, rhoR, pR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def sample(xi, rhoL, uL, pL, rhoR, uR, pR, g):
    """(rho, u, p) at similarity coordinate xi = (x - x0)/t (array)."""
    xi = np.asarray(xi, dtype=np.float64)
    ps, us = star_state(rhoL, uL, pL, rhoR, uR, pR, g)
    aL = math.sqrt(g * pL / rhoL)
    aR = math.sqrt(g * pR / rhoR)
    gm = (g - 1.0) / (g + 1.0)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for i, s in enumerate(xi.ravel()):
        if s <= us:  # left of the contact
            if ps > pL:  # left shock
                SL = uL - aL * math.sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
                if s <= SL:
                    r, v, q = rhoL, uL, pL
                else:
                    r = rhoL * ((ps / pL + gm) / (gm * ps / pL + 1.0))
                    v, q = us, ps
            else:  # left rarefaction
                aLs = aL * (ps / pL) ** ((g - 1.0) / (2.0 * g))
                head, tail = uL - aL, us - aLs
                if s <= head:
                    r, v, q = rhoL, uL, pL
                elif s >= tail:
                    r, v, q = rhoL * (ps / pL) ** (1.0 / g), us, ps
                else:
                    c = 2.0 / (g + 1.0) + gm / aL * (uL - s)
                    r = rhoL * c ** (2.0 / (g - 1.0))
                    v = 2.0 / (g + 1.0) * (aL + (g - 1.0) / 2.0 * uL + s)
                    q = pL * c ** (2.0 * g / (g - 1.0))
        else:  # right of the contact
            if ps > pR:  # right shock
                SR = uR + aR * math.sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
                if s >= SR:
                    r, v, q = rhoR, uR, pR
                else:
                    r = rhoR * ((ps / pR + gm) / (gm * ps / pR + 1.0))
                    v, q = us, ps
            else:  # right rarefaction
                aRs = aR * (ps / pR) ** ((g - 1.0) / (2.0 * g))
                head, tail = uR + aR, us + aRs
                if s >= head:
                    r, v, q = rhoR, uR, pR
                elif s <= tail:
                    r, v, q = rhoR * (ps / pR) ** (1.0 / g), us, ps
                else:
                    c = 2.0 / (g + 1.0) - gm / aR * (uR - s)
                    r = rhoR * c ** (2.0 / (g - 1.0))
                    v = 2.0 / (g + 1.0) * (-aR + (g - 1.0) / 2.0 * uR + s)
                    q = pR * c ** (2.0 * g / (g - 1.0))
        rho.flat[i], u.flat[i], p.flat[i] = r, v, q
    return rho, u, p
