"""Exact solution of the 1-D Riemann problem for an ideal gas.

TEST INFRASTRUCTURE ONLY (part of the oracle).  The paper (Sec. V) compares
its shock-tube runs with "the analytical solution" without printing it; this
is the standard exact solver (the two-wave pressure function of Godunov's
method: a shock or a rarefaction on each side of a contact, the star-state
pressure found by Newton's method, then sampled along x/t), written for the
non-dimensional units of Sec. II, where p = rho T and the sound speed is
a = sqrt(gamma p / rho).
"""
from __future__ import annotations

import math

import numpy as np


def _wave(p, rho_k, p_k, a_k, gamma):
    """Velocity jump f_k(p) across the left/right wave and its derivative."""
    if p > p_k:  # shock
        A = 2.0 / ((gamma + 1.0) * rho_k)
        B = (gamma - 1.0) / (gamma + 1.0) * p_k
        q = math.sqrt(A / (p + B))
        f = (p - p_k) * q
        df = q * (1.0 - 0.5 * (p - p_k) / (B + p))
    else:  # rarefaction
        e = (gamma - 1.0) / (2.0 * gamma)
        f = 2.0 * a_k / (gamma - 1.0) * ((p / p_k) ** e - 1.0)
        df = 1.0 / (rho_k * a_k) * (p / p_k) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma):
    """(p*, u*) between the waves.  left/right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    al = math.sqrt(gamma * pl / rl)
    ar = math.sqrt(gamma * pr / rr)
    if 2.0 * (al + ar) / (gamma - 1.0) <= ur - ul:
        raise ValueError("vacuum is generated; not a shock-tube state")
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _wave(p, rl, pl, al, gamma)
        fr, dfr = _wave(p, rr, pr, ar, gamma)
        g = fl + fr + ur - ul
        dp = g / (dfl + dfr)
        p_new = max(1e-14, p - dp)
        if abs(p_new - p) <= 1e-15 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _wave(p, rl, pl, al, gamma)
    fr, _ = _wave(p, rr, pr, ar, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, gamma, xi):
    """(rho, u, p) at similarity coordinates xi = (x - x0) / t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    al = math.sqrt(gamma * pl / rl)
    ar = math.sqrt(gamma * pr / rr)
    ps, us = star_state(left, right, gamma)
    gm = (gamma - 1.0) / (gamma + 1.0)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for k, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                rs = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                sl = ul - al * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl
                                         + (gamma - 1.0) / (2.0 * gamma))
                vals = (rl, ul, pl) if s <= sl else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / gamma)
                a_s = al * (ps / pl) ** ((gamma - 1.0) / (2.0 * gamma))
                head, tail = ul - al, us - a_s
                if s <= head:
                    vals = (rl, ul, pl)
                elif s >= tail:
                    vals = (rs, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) + gm / al * (ul - s)
                    vals = (rl * c ** (2.0 / (gamma - 1.0)),
                            2.0 / (gamma + 1.0) * (al + 0.5 * (gamma - 1.0) * ul + s),
                            pl * c ** (2.0 * gamma / (gamma - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                rs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                sr = ur + ar * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr
                                         + (gamma - 1.0) / (2.0 * gamma))
                vals = (rs, us, ps) if s <= sr else (rr, ur, pr)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / gamma)
                a_s = ar * (ps / pr) ** ((gamma - 1.0) / (2.0 * gamma))
                head, tail = ur + ar, us + a_s
                if s >= head:
                    vals = (rr, ur, pr)
                elif s <= tail:
                    vals = (rs, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) - gm / ar * (ur - s)
                    vals = (rr * c ** (2.0 / (gamma - 1.0)),
                            2.0 / (gamma + 1.0) * (-ar + 0.5 * (gamma - 1.0) * ur + s),
                            pr * c ** (2.0 * gamma / (gamma - 1.0)))
        rho[k], u[k], p[k] = vals
    return rho, u, p


def shock_tube_profile(left, right, gamma, nx, t, x0=0.5):
    """Exact (rho, u, T) at the cell centres x_j = (j + 1/2)/nx of [0, 1] at
    time t; the diaphragm sits at x0.  left/right = (rho, u, p)."""
    x = (np.arange(nx) + 0.5) / nx
    rho, u, p = sample(left, right, gamma, (x - x0) / t)
    return rho, u, p / rho


def lattice_time(steps, nx, r):
    """Physical time of a lattice run (Sec. V): t = steps / (X r)."""
    return steps / (nx * r)


def l1_error(q, q_exact, cells=None):
    """Mean absolute error per cell, optionally over a cell slice."""
    q = np.asarray(q)
    q_exact = np.asarray(q_exact)
    if cells is not None:
        q = q[cells]
        q_exact = q_exact[cells]
    return float(np.mean(np.abs(q - q_exact)))
