"""Exact solutions used to pin the oracle (test infrastructure only).

* `sod_exact`: the exact Riemann solution of the Euler equations for an ideal gas, the
  reference of the paper's Sod tube (Sec. 3.2, Tab. sod_conv).  Star pressure by Newton
  iteration on f_L(p) + f_R(p) + (u_R - u_L) = 0 with the shock (Rankine-Hugoniot) and
  rarefaction (isentropic) branches of f_K; self-similar sampling in xi = (x - x0)/t.
* `becker_profile`: Becker's closed-form viscous shock (Sec. 3.2) for constant mu and
  Pr = 3/4.  With Pr = 3/4 the total enthalpy H = c_p T + u^2/2 is constant through the
  front, and v = u/u1 obeys dv/dx = K (v - 1)(v - v2)/v, K = 3 (gamma+1) rho1 u1 / (8 gamma mu),
  v2 = (gamma-1)/(gamma+1) + 2/((gamma+1) M^2); integrated:
      ln(1 - v) - v2 ln(v - v2) = (1 - v2) K (x - x0) + C,
  with C fixing v(x0) = (1 + v2)/2.  The implicit relation is inverted by bisection.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, ck, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (B + p))
    e = (g - 1.0) / (2.0 * g)
    f = 2.0 * ck / (g - 1.0) * ((p / pk) ** e - 1.0)
    d = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, d


def sod_star(left, right, gamma=1.4):
    """Star-region pressure and velocity for left/right (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _fk(p, rl, pl, cl, gamma)
        fr, dr = _fk(p, rr, pr, cr, gamma)
        f = fl + fr + (ur - ul)
        pn = max(1e-12, p - f / (dl + dr))
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, gamma)
    fr, _ = _fk(p, rr, pr, cr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sod_exact(x, t, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x0=0.5, gamma=1.4):
    """Exact (rho, u, p) at positions x and time t > 0."""
    g = gamma
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    ps, us = sod_star(left, right, g)
    G6 = (g - 1.0) / (g + 1.0)
    x = np.asarray(x, np.float64)
    out = np.zeros((3, x.size))
    for n, xi in enumerate(((x - x0) / t).ravel()):
        if xi <= us:
            if ps > pl:  # left shock
                SL = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if xi <= SL:
                    w = (rl, ul, pl)
                else:
                    w = (rl * (ps / pl + G6) / (G6 * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                SHL = ul - cl
                cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
                STL = us - cs
                if xi <= SHL:
                    w = (rl, ul, pl)
                elif xi >= STL:
                    w = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) * (cl + 0.5 * (g - 1) * (ul - xi))
                    u = 2.0 / (g + 1) * (cl + 0.5 * (g - 1) * ul + xi)
                    w = (rl * (c / cl) ** (2 / (g - 1)), u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:
            if ps > pr:  # right shock
                SR = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if xi >= SR:
                    w = (rr, ur, pr)
                else:
                    w = (rr * (ps / pr + G6) / (G6 * ps / pr + 1.0), us, ps)
            else:  # right rarefaction
                SHR = ur + cr
                cs = cr * (ps / pr) ** ((g - 1) / (2 * g))
                STR = us + cs
                if xi >= SHR:
                    w = (rr, ur, pr)
                elif xi <= STR:
                    w = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) * (cr - 0.5 * (g - 1) * (ur - xi))
                    u = 2.0 / (g + 1) * (-cr + 0.5 * (g - 1) * ur + xi)
                    w = (rr * (c / cr) ** (2 / (g - 1)), u, pr * (c / cr) ** (2 * g / (g - 1)))
        out[:, n] = w
    return out[0], out[1], out[2]


def becker_v2(mach, gamma=1.4):
    return (gamma - 1.0) / (gamma + 1.0) + 2.0 / ((gamma + 1.0) * mach * mach)


def becker_profile(x, mach, mu, x0, gamma=1.4, rho1=1.0, c1=1.0):
    """Stationary Becker shock (flow in +x, upstream at x -> -inf).  Returns rho, u, p."""
    g = gamma
    u1 = mach * c1
    p1 = rho1 * c1 * c1 / g
    T1 = p1 / rho1
    cp = g / (g - 1.0)
    H = cp * T1 + 0.5 * u1 * u1
    v2 = becker_v2(mach, g)
    K = 3.0 * (g + 1.0) * rho1 * u1 / (8.0 * g * mu)
    vm = 0.5 * (1.0 + v2)
    C0 = math.log(1.0 - vm) - v2 * math.log(vm - v2)
    rhs = (1.0 - v2) * K * (np.asarray(x, np.float64) - x0) + C0
    # G(v) = ln(1-v) - v2 ln(v - v2) is strictly decreasing on (v2, 1): bisection
    lo = np.full(rhs.shape, v2)
    hi = np.ones(rhs.shape)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        Gm = np.log(np.maximum(1.0 - mid, 1e-300)) - v2 * np.log(np.maximum(mid - v2, 1e-300))
        big = Gm > rhs          # G too large -> v too small
        lo = np.where(big, mid, lo)
        hi = np.where(big, hi, mid)
    v = 0.5 * (lo + hi)
    u = u1 * v
    rho = rho1 / v
    T = (H - 0.5 * u * u) / cp
    return rho, u, rho * T
