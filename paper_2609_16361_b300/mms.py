"""Manufactured solution of Sec. 3.1 (Eq. mms): exact fields and the source that makes them
solve the compressible Navier-Stokes-Fourier system (Eq. system), as problem inputs.

The source is S = d_t Q + div Phi(Q) with the full flux (Newtonian stress, Fourier flux,
constant mu and kappa = mu c_p / Pr) evaluated symbolically on the manufactured primitives and
lambdified for numpy (or torch).  It defines the problem, like an initial field; it holds no
lattice Boltzmann arithmetic.

Reading of the scales (Sec. 3.1 and Tab. run_params): unit periodic box, k = 2 pi, unit
temporal period, rho0 = 1, velocity scale c_s = 1, a = 0.30/sqrt(3), p0 = rho0 c_s^2
(0.30/M0)^2/gamma with M0 = 2; acoustic refinement dt = 0.05 dx; BGK with the dt-tied
relaxation: tau - 1/2 proportional to dt, omega = 1.86 at the finest grid N = 256 (a fixed
omega leaves a numerical diffusivity cs^2 (tau - 1/2) dx^2/dt proportional to dx, i.e. first
order); the viscosity is fixed so that beta = 2 nu_lat omega / cs^2 is about 0.5 at N = 64
(mu = 0.0105), growing with N as the paper states.
"""
from __future__ import annotations

import functools
import math

import numpy as np

from . import inputs

GAMMA = 1.4
M0 = 2.0
RHO0 = 1.0
CS = 1.0
A = 0.30 / math.sqrt(3.0)
P0 = RHO0 * CS ** 2 * (0.30 / M0) ** 2 / GAMMA
MU = 0.0105
PR = 0.71
OMEGA = 1.86
FINE_N = 256
CFL = 0.05


def omega_tied(n):
    """dt-tied relaxation: tau - 1/2 proportional to dt (to dx), omega = OMEGA at FINE_N."""
    return 1.0 / (0.5 + (1.0 / OMEGA - 0.5) * FINE_N / n)


@functools.lru_cache(maxsize=None)
def _symbolic(mu=MU, pr=PR, gamma=GAMMA):
    import sympy as sp
    x, y, z, t = sp.symbols("x y z t", real=True)
    k = 2 * sp.pi
    w = 2 * sp.pi
    rho = RHO0 * (1 + sp.Rational(5, 100) * sp.sin(k * x) + sp.Rational(3, 100) * sp.cos(k * y)
                  + sp.Rational(2, 100) * sp.cos(k * z + w * t))
    ux = CS * (A + sp.Rational(35, 1000) * sp.cos(k * x + sp.Rational(4, 10))
               + sp.Rational(25, 1000) * sp.sin(k * y))
    uy = CS * (A + sp.Rational(35, 1000) * sp.sin(k * y + sp.Rational(9, 10))
               + sp.Rational(25, 1000) * sp.cos(k * z))
    uz = CS * (A + sp.Rational(25, 1000) * sp.cos(k * z + sp.Rational(17, 10))
               + sp.Rational(15, 1000) * sp.sin(k * x + w * t))
    p = P0 * (1 + sp.Rational(5, 100) * sp.cos(k * x + sp.Rational(12, 10))
              + sp.Rational(3, 100) * sp.sin(k * y + w * t) + sp.Rational(2, 100) * sp.sin(k * z + sp.Rational(6, 10)))
    X = [x, y, z]
    u = [ux, uy, uz]
    T = p / rho
    E = p / (gamma - 1) + sp.Rational(1, 2) * rho * (ux ** 2 + uy ** 2 + uz ** 2)
    cp = gamma / (gamma - 1)
    kappa = mu * cp / pr
    div = sum(sp.diff(u[j], X[j]) for j in range(3))
    tau = [[mu * (sp.diff(u[a], X[b]) + sp.diff(u[b], X[a]) - (sp.Rational(2, 3) * div if a == b else 0))
            for b in range(3)] for a in range(3)]
    q = [-kappa * sp.diff(T, X[c]) for c in range(3)]
    Q = [rho, rho * ux, rho * uy, rho * uz, E]
    flux = [[rho * u[c] for c in range(3)]]
    for j in range(3):
        flux.append([rho * u[j] * u[c] + (p if j == c else 0) - tau[j][c] for c in range(3)])
    flux.append([(E + p) * u[c] - sum(tau[c][b] * u[b] for b in range(3)) + q[c] for c in range(3)])
    S = [sp.diff(Q[kk], t) + sum(sp.diff(flux[kk][c], X[c]) for c in range(3)) for kk in range(5)]
    return (x, y, z, t), (rho, ux, uy, uz, p), S


@functools.lru_cache(maxsize=None)
def _lambdas(module="numpy", mu=MU, pr=PR):
    import sympy as sp
    args, prim, S = _symbolic(mu, pr)
    fprim = sp.lambdify(args, prim, modules=module, cse=True)
    fsrc = sp.lambdify(args, S, modules=module, cse=True)
    return fprim, fsrc


def grid(n):
    c = (np.arange(n, dtype=np.float64) + 0.5) / n
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def _bcast(v, shape):
    return np.broadcast_to(np.asarray(v, dtype=np.float64), shape).copy()


def primitive(n, t):
    """Exact rho, u (3, N), p at cell centres of the n^3 grid at time t."""
    X, Y, Z = grid(n)
    rho, ux, uy, uz, p = _lambdas()[0](X, Y, Z, t)
    sh = X.shape
    return _bcast(rho, sh), np.stack([_bcast(ux, sh), _bcast(uy, sh), _bcast(uz, sh)]), _bcast(p, sh)


def conserved(n, t):
    rho, u, p = primitive(n, t)
    return np.stack([rho, rho * u[0], rho * u[1], rho * u[2],
                     p / (GAMMA - 1) + 0.5 * rho * (u * u).sum(0)])


def source(n, t):
    """S_k(x, t) (5, N) in physical units: rates of (rho, m_x, m_y, m_z, E) per unit time."""
    X, Y, Z = grid(n)
    S = _lambdas()[1](X, Y, Z, t)
    return np.stack([_bcast(s, X.shape) for s in S])


def case(n, storage=inputs.STORE_F32) -> inputs.Case:
    """Initial state (t = 0) and parameters of the manufactured-solution run at n^3."""
    dx = 1.0 / n
    dt = CFL * dx
    rho, u, p = primitive(n, 0.0)
    om = omega_tied(n)
    prm = inputs.CaseParams(nx=n, ny=n, nz=n, bc=inputs.BC_PERIODIC, collision=inputs.COLL_BGK,
                            storage=storage, dx=dx, dt=dt, gamma=GAMMA, mu_ref=MU, prandtl=PR,
                            T_ref=P0 / RHO0, sutherland=0, omega_rho=om, omega_mom=om,
                            omega_E=om, omega_min=1.0, sensor_gain=0.0, J_min=1.0,
                            rho_min=1e-4, p_min=1e-6, ref_rho=RHO0, ref_p=P0, name=f"mms{n}")
    return inputs.Case(prm, rho, u, p, dict(dt=dt, dx=dx))
