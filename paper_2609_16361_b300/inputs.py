"""Synthetic case generators shared by the CUDA path and the FP64 oracle.

This module only builds inputs: a physical-unit parameter record and primitive initial
fields (rho, u, p) on the grid, x fastest.  It holds none of the scheme's arithmetic (no
lattice conversion, no equilibrium, no collision); each side does that itself.

Cases follow the paper's workloads:
  * Sod shock tube (Sec. 3.2, Tab. run_params): gamma = 1.4, (1, 0, 1) | (0.125, 0, 0.1).
  * Becker viscous shock (Sec. 3.2): constant mu, Pr = 3/4, stationary shock frame.
  * Compressible Taylor-Green vortex (Sec. 3.4): Re = 1600, M0 = 1.25, Sutherland law,
    background damping f_mu per resolution, tau = 1/2 + 4 f_mu nu dt/dx^2.
  * uniform states, low-Mach 2-D Taylor-Green decay, seeded smooth random fields.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

BC_PERIODIC = 0
BC_X_DIRICHLET_EQ = 1
COLL_BGK = 0
COLL_RLB_SENSOR = 1
COLL_RLB_GATED = 2   # BGK where the sensor is off, regularized where it fires
STORE_F32 = 0
STORE_F16 = 1
STORE_BF16 = 2

SUTHERLAND_TS = 0.4042  # Listing 1


@dataclass
class CaseParams:
    """Physical-unit description of one domain (mirrors the C struct grlb_params)."""

    nx: int
    ny: int
    nz: int
    bc: int = BC_PERIODIC
    collision: int = COLL_RLB_SENSOR
    storage: int = STORE_F32
    streaming: int = 0        # 0: two buffers (pull), 1: one buffer, AA pattern, 2: two buffers of
                              # moments (FP32 storage, regularized collision)
    dx: float = 1.0
    dt: float = 1.0
    gamma: float = 1.4
    mu_ref: float = 0.0
    prandtl: float = 0.71
    T_ref: float = 1.0
    sutherland: int = 0
    T_S: float = SUTHERLAND_TS
    omega_rho: float = 1.9
    omega_mom: float = 1.9
    omega_E: float = 1.9
    omega_min: float = 1.0
    sensor_gain: float = 20.0
    J_min: float = 3e-3
    rho_min: float = 1e-4
    p_min: float = 1e-4
    ref_rho: float = 1.0
    ref_p: float = 1.0
    left_prim: tuple = (1.0, 0.0, 0.0, 0.0, 1.0)
    right_prim: tuple = (1.0, 0.0, 0.0, 0.0, 1.0)
    name: str = "case"

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "CaseParams":
        return dataclasses.replace(self, **kw)


@dataclass
class Case:
    params: CaseParams
    rho: np.ndarray            # (N,) float64, x fastest
    u: np.ndarray              # (3, N) float64
    p: np.ndarray              # (N,) float64
    meta: dict = field(default_factory=dict)


def _grid(n, d, offset):
    return (np.arange(n, dtype=np.float64) + offset) * d


def _flat(a):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


# --------------------------------------------------------------------------------------
def fmu_for_resolution(n: int) -> float:
    """Background damping f_mu of Sec. 3.4 (1.8, 0.9, 0.001, 0.01 at 64^3..512^3); other
    sizes take the nearest listed resolution on a log scale."""
    table = [(64, 1.8), (128, 0.9), (256, 0.001), (512, 0.01)]
    return min(table, key=lambda t: abs(math.log(n / t[0])))[1]


def tgv3d(n: int, mach: float = 1.25, re: float = 1600.0, pr: float = 0.71,
          cfl: float = 0.1, fmu: float | None = None, storage: int = STORE_F32,
          collision: int = COLL_RLB_SENSOR, sutherland: int = 1, nxyz=None,
          omega_min: float = 1.987) -> Case:
    """Compressible Taylor-Green vortex on [0, 2 pi)^3 with V0 = L0 = rho0 = 1.

    Velocity u = V0 sin x cos y cos z, v = -V0 cos x sin y cos z, w = 0; pressure
    p = p0 + rho0 V0^2/16 (cos 2x + cos 2y)(cos 2z + 2) with p0 = rho0 V0^2 / (gamma M0^2);
    density rho = p / T0 at uniform temperature T0 = p0/rho0.  dt = cfl * dx.
    nxyz overrides the grid extent (a slab of the n^3 problem with identical per-cell
    parameters), used for bounded CPU samples.  omega_min: the sensor floor rate (Tab.
    run_params: 1.987; 1.8 is the nearest setting at which the regularized collision stays
    finite to t_c 20)."""
    gamma = 1.4
    nx, ny, nz = nxyz if nxyz is not None else (n, n, n)
    dx = 2.0 * math.pi / n
    dt = cfl * dx
    V0 = 1.0
    rho0 = 1.0
    p0 = rho0 * V0 * V0 / (gamma * mach * mach)
    T0 = p0 / rho0
    mu = rho0 * V0 * 1.0 / re
    if fmu is None:
        fmu = fmu_for_resolution(n)
    nu_lat = mu / rho0 * dt / (dx * dx)
    tau = 0.5 + 4.0 * fmu * nu_lat
    omega = 1.0 / tau
    x = _grid(nx, dx, 0.0)
    y = _grid(ny, dx, 0.0)
    z = _grid(nz, dx, 0.0)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    ux = V0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    uy = -V0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    uz = np.zeros_like(ux)
    p = p0 + rho0 * V0 * V0 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    rho = p / T0
    prm = CaseParams(nx=nx, ny=ny, nz=nz, bc=BC_PERIODIC, collision=collision, storage=storage,
                     dx=dx, dt=dt, gamma=gamma, mu_ref=mu, prandtl=pr, T_ref=T0,
                     sutherland=sutherland, omega_rho=omega, omega_mom=omega, omega_E=omega,
                     omega_min=omega_min, sensor_gain=40.0, J_min=1e-2, rho_min=1e-4, p_min=1e-4,
                     ref_rho=rho0, ref_p=p0, name=f"tgv{n}")
    meta = dict(V0=V0, L0=1.0, rho0=rho0, p0=p0, T0=T0, mach=mach, re=re, fmu=fmu,
                tc_per_step=dt * V0 / 1.0)
    return Case(prm, _flat(rho), np.stack([_flat(ux), _flat(uy), _flat(uz)]), _flat(p), meta)


def tgv3d_device(n: int, device="cuda", **kw):
    """tgv3d(n, **kw) with its fields built on the device, one z-plane at a time, as torch FP64
    tensors (rho (N,), u (3, N), p (N,)): for domains whose n^3 host arrays would not fit the
    host.  Returns (params, rho, u, p); the same formulas as tgv3d."""
    import torch
    c = tgv3d(n, nxyz=(n, n, 1), **kw)  # the n^3 case's parameters, one plane of fields
    prm = c.params.replace(nz=n)
    m = c.meta
    N = n * n * n
    f64 = dict(dtype=torch.float64, device=device)
    rho = torch.empty(N, **f64)
    u = torch.empty((3, N), **f64)
    p = torch.empty(N, **f64)
    x = (torch.arange(n, **f64) + 0.0) * prm.dx
    X, Y = x[None, :], x[:, None]
    for z in range(n):
        Z = torch.tensor(z * prm.dx, **f64)
        sl = slice(z * n * n, (z + 1) * n * n)
        u[0, sl] = (m["V0"] * torch.sin(X) * torch.cos(Y) * torch.cos(Z)).reshape(-1)
        u[1, sl] = (-m["V0"] * torch.cos(X) * torch.sin(Y) * torch.cos(Z)).reshape(-1)
        u[2, sl] = 0.0
        pz = m["p0"] + m["rho0"] * m["V0"] ** 2 / 16.0 * (torch.cos(2 * X) + torch.cos(2 * Y)) * (torch.cos(2 * Z) + 2.0)
        p[sl] = pz.reshape(-1)
        rho[sl] = p[sl] / m["T0"]
    return prm, rho, u, p


def sod(nx: int = 400, t_end: float = 0.2, steps: int = 1000, storage: int = STORE_F32,
        mu: float = 1e-6, omega: float = 1.40) -> Case:
    """Sod tube on [0, 1], diaphragm between cells nx/2 - 1 and nx/2 (x = 0.5).
    dt = t_end / steps; with 400 cells and 1000 steps dt/dx = 0.08."""
    gamma = 1.4
    dx = 1.0 / nx
    dt = t_end / steps
    left = (1.0, 0.0, 0.0, 0.0, 1.0)
    right = (0.125, 0.0, 0.0, 0.0, 0.1)
    xi = np.arange(nx)
    rho = np.where(xi < nx // 2, left[0], right[0]).astype(np.float64)
    p = np.where(xi < nx // 2, left[4], right[4]).astype(np.float64)
    u = np.zeros((3, nx))
    prm = CaseParams(nx=nx, ny=1, nz=1, bc=BC_X_DIRICHLET_EQ, collision=COLL_RLB_SENSOR,
                     storage=storage, dx=dx, dt=dt, gamma=gamma, mu_ref=mu, prandtl=0.71,
                     T_ref=1.0, sutherland=0, omega_rho=omega, omega_mom=omega, omega_E=omega,
                     omega_min=1.0, sensor_gain=20.0, J_min=3e-3, rho_min=1e-4, p_min=1e-4,
                     ref_rho=0.5, ref_p=0.5, left_prim=left, right_prim=right,
                     name=f"sod{nx}")
    return Case(prm, rho, u, p, dict(t_end=t_end, steps=steps, x=(xi + 0.5) * dx))


def double_rarefaction(nx: int = 400, t_end: float = 0.15, steps: int = 750, p_min: float = 0.01,
                       storage: int = STORE_F32, omega: float = 1.40) -> Case:
    """Toro's test 2 (two strong rarefactions, near-vacuum star state p* = 0.00189,
    rho* = 0.0219): (rho, u, p) = (1, -2, 0.4) | (1, 2, 0.4) on [0, 1], diaphragm at x = 0.5,
    shock-tube settings of Tab. run_params (RLB, omega 1.40, g 20, J_min 3e-3, omega_min 1).
    The pressure floor p_min (physical units) is raised above p* so that the positivity floor
    of Alg. 1 acts in the star region.  dt = t_end / steps; 400 cells and 750 steps give
    dt/dx = 0.08 and max(|u| + c) dt/dx = 0.22."""
    gamma = 1.4
    dx = 1.0 / nx
    dt = t_end / steps
    left = (1.0, -2.0, 0.0, 0.0, 0.4)
    right = (1.0, 2.0, 0.0, 0.0, 0.4)
    xi = np.arange(nx)
    rho = np.ones(nx)
    p = np.full(nx, 0.4)
    u = np.zeros((3, nx))
    u[0] = np.where(xi < nx // 2, left[1], right[1])
    prm = CaseParams(nx=nx, ny=1, nz=1, bc=BC_X_DIRICHLET_EQ, collision=COLL_RLB_SENSOR,
                     storage=storage, dx=dx, dt=dt, gamma=gamma, mu_ref=1e-6, prandtl=0.71,
                     T_ref=1.0, sutherland=0, omega_rho=omega, omega_mom=omega, omega_E=omega,
                     omega_min=1.0, sensor_gain=20.0, J_min=3e-3, rho_min=1e-4, p_min=p_min,
                     ref_rho=0.5, ref_p=0.2, left_prim=left, right_prim=right,
                     name=f"toro2_{nx}")
    return Case(prm, rho, u, p, dict(t_end=t_end, steps=steps, x=(xi + 0.5) * dx))


def becker_states(mach: float, gamma: float = 1.4):
    """Upstream (rho1=1, c1=1, u1=M) and Rankine-Hugoniot downstream state of a stationary
    normal shock.  Returns ((rho, u, p) upstream, (rho, u, p) downstream)."""
    rho1, c1 = 1.0, 1.0
    p1 = rho1 * c1 * c1 / gamma
    u1 = mach * c1
    r = (gamma + 1.0) * mach ** 2 / ((gamma - 1.0) * mach ** 2 + 2.0)
    rho2 = rho1 * r
    u2 = u1 / r
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (mach ** 2 - 1.0))
    return (rho1, u1, p1), (rho2, u2, p2)


def becker(nx: int, mach: float = 2.0, cells_per_front: float = 8.0, cfl_max: float = 0.3,
           ny: int = 1, nz: int = 1, omega: float = 1.99, storage: int = STORE_F32,
           x_shock: float = 0.5) -> Case:
    """Stationary Becker viscous shock on [0, 1] with Pr = 3/4 and constant mu.

    mu is set so that the velocity front (u1 - u2)/max|u'| spans `cells_per_front` cells;
    dt is set so that max(|u| + c) * dt/dx = cfl_max.  Initial field: tanh profile of the
    front width between the Rankine-Hugoniot states (the scheme forms its own structure).
    Ends are equilibrium ghosts at the upstream / downstream states."""
    gamma = 1.4
    (r1, u1, p1), (r2, u2, p2) = becker_states(mach, gamma)
    dx = 1.0 / nx
    # front width of the Becker profile: delta = (1 - v2) / max_v[K (1-v)(v-v2)/v] in x*u1-units
    v2 = u2 / u1
    vv = np.linspace(v2, 1.0, 20001)[1:-1]
    shape = np.max((1.0 - vv) * (vv - v2) / vv)
    # K = 3 (gamma+1) rho1 u1 / (8 gamma mu); delta = (1 - v2) / (K * shape)
    delta = cells_per_front * dx
    mu = 3.0 * (gamma + 1.0) * r1 * u1 * shape * delta / (8.0 * gamma * (1.0 - v2))
    c1 = math.sqrt(gamma * p1 / r1)
    c2 = math.sqrt(gamma * p2 / r2)
    smax = max(u1 + c1, u2 + c2)
    dt = cfl_max * dx / smax
    x = (np.arange(nx) + 0.5) * dx
    w = 0.5 * (1.0 + np.tanh((x - x_shock) / (0.5 * delta)))
    rho = r1 + (r2 - r1) * w
    ux = u1 + (u2 - u1) * w
    p = p1 + (p2 - p1) * w
    rho = np.tile(rho, ny * nz)
    ux = np.tile(ux, ny * nz)
    p = np.tile(p, ny * nz)
    u = np.stack([ux, np.zeros_like(ux), np.zeros_like(ux)])
    prm = CaseParams(nx=nx, ny=ny, nz=nz, bc=BC_X_DIRICHLET_EQ, collision=COLL_RLB_SENSOR,
                     storage=storage, dx=dx, dt=dt, gamma=gamma, mu_ref=mu, prandtl=0.75,
                     T_ref=1.0, sutherland=0, omega_rho=omega, omega_mom=omega,
                     omega_E=omega, omega_min=1.0, sensor_gain=20.0, J_min=3e-3,
                     rho_min=1e-4, p_min=1e-4, ref_rho=0.5 * (r1 + r2),
                     ref_p=0.5 * (p1 + p2), left_prim=(r1, u1, 0.0, 0.0, p1),
                     right_prim=(r2, u2, 0.0, 0.0, p2), name=f"becker{nx}")
    meta = dict(mach=mach, mu=mu, delta=delta, x=x, x_shock=x_shock,
                up=(r1, u1, p1), down=(r2, u2, p2))
    return Case(prm, rho, u, p, meta)


def uniform(nx: int, ny: int, nz: int, rho=1.0, u=(0.05, -0.03, 0.02), p=0.6,
            collision: int = COLL_RLB_SENSOR, storage: int = STORE_F32,
            sutherland: int = 1) -> Case:
    """Uniform state at rest in a moving frame; invariant under the exact scheme."""
    N = nx * ny * nz
    prm = CaseParams(nx=nx, ny=ny, nz=nz, bc=BC_PERIODIC, collision=collision,
                     storage=storage, dx=1.0, dt=0.5, gamma=1.4, mu_ref=2e-3, prandtl=0.71,
                     T_ref=p / rho, sutherland=sutherland, omega_rho=1.95, omega_mom=1.95,
                     omega_E=1.95, omega_min=1.5, sensor_gain=20.0, J_min=3e-3,
                     ref_rho=rho, ref_p=p, name="uniform")
    return Case(prm, np.full(N, float(rho)), np.tile(np.asarray(u, float)[:, None], (1, N)),
                np.full(N, float(p)))


def tgv2d(n: int, mach: float = 0.05, nu_lat: float = 0.01, omega: float = 2.0,
          collision: int = COLL_BGK) -> Case:
    """Low-Mach 2-D Taylor-Green vortex on an n x n x 1 periodic box (unit box L = 1).

    u = V0 sin(kx) cos(ky), v = -V0 cos(kx) sin(ky), k = 2 pi; p = p0 + rho0 V0^2/4
    (cos 2kx + cos 2ky), rho = p/T0.  Incompressible kinetic energy decays as
    exp(-4 nu k^2 t); constant mu with nu = mu / rho0."""
    gamma = 1.4
    dx = 1.0 / n
    V0 = 1.0
    rho0 = 1.0
    c0 = V0 / mach
    p0 = rho0 * c0 * c0 / gamma
    T0 = p0 / rho0
    # lattice velocity scale: keep max(|u| + c) dt/dx = 0.15
    dt = 0.15 * dx / (V0 + c0)
    nu = nu_lat * dx * dx / dt
    mu = rho0 * nu
    k = 2.0 * math.pi
    x = _grid(n, dx, 0.5)
    Y, X = np.meshgrid(x, x, indexing="ij")
    ux = V0 * np.sin(k * X) * np.cos(k * Y)
    uy = -V0 * np.cos(k * X) * np.sin(k * Y)
    p = p0 + rho0 * V0 * V0 / 4.0 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    rho = p / T0
    prm = CaseParams(nx=n, ny=n, nz=1, bc=BC_PERIODIC, collision=collision, dx=dx, dt=dt,
                     gamma=gamma, mu_ref=mu, prandtl=0.71, T_ref=T0, sutherland=0,
                     omega_rho=omega, omega_mom=omega, omega_E=omega, omega_min=1.0,
                     sensor_gain=20.0, J_min=3e-3, ref_rho=rho0, ref_p=p0, name=f"tgv2d{n}")
    u = np.stack([_flat(ux), _flat(uy), np.zeros(n * n)])
    return Case(prm, _flat(rho), u, _flat(p), dict(nu=nu, k=k, V0=V0, rho0=rho0))


def random_smooth(nx: int, ny: int, nz: int, seed: int = 0, amp: float = 0.05,
                  mach: float = 0.5, collision: int = COLL_RLB_SENSOR, sutherland: int = 1,
                  storage: int = STORE_F32) -> Case:
    """Seeded smooth random periodic field: a few low Fourier modes per primitive."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / max(nx, ny, nz)
    x = _grid(nx, dx, 0.0)
    y = _grid(ny, dx, 0.0)
    z = _grid(nz, dx, 0.0)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    Lx, Ly, Lz = nx * dx, ny * dx, nz * dx

    def modes(scale):
        out = np.zeros_like(X)
        for _ in range(4):
            kx, ky, kz = rng.integers(0, 3, size=3)
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-0.25, 0.25) * scale
            out += a * np.cos(2 * math.pi * (kx * X / Lx + ky * Y / Ly + kz * Z / Lz) + ph)
        return out

    rho0, p0 = 1.0, 1.0 / 1.4
    c0 = 1.0
    V = mach * c0
    rho = rho0 * (1.0 + modes(amp))
    p = p0 * (1.0 + modes(amp))
    ux, uy, uz = V * modes(1.0), V * modes(1.0), V * modes(1.0)
    dt = 0.25 * dx / (V + c0)
    prm = CaseParams(nx=nx, ny=ny, nz=nz, bc=BC_PERIODIC, collision=collision, storage=storage,
                     dx=dx, dt=dt, gamma=1.4, mu_ref=5e-4, prandtl=0.71, T_ref=p0 / rho0,
                     sutherland=sutherland, omega_rho=1.97, omega_mom=1.97, omega_E=1.97,
                     omega_min=1.9, sensor_gain=40.0, J_min=1e-2, ref_rho=rho0, ref_p=p0,
                     name=f"rand{seed}")
    return Case(prm, _flat(rho), np.stack([_flat(ux), _flat(uy), _flat(uz)]), _flat(p))


# --------------------------------------------------------------------------------------
# Multi-domain workloads (seeded)
def becker_tied_omega(cells_per_front: float, fine_cells: float = 128.0, fine_omega: float = 1.99):
    """omega tied to dt: tau - 1/2 proportional to dt (cells_per_front under acoustic scaling),
    equal to fine_omega at fine_cells cells per front."""
    return 1.0 / (0.5 + (1.0 / fine_omega - 0.5) * fine_cells / cells_per_front)


def batched_mix(seed: int = 0, n_becker: int = 48, n_tgv: int = 16, storage: int = STORE_F32):
    """Uneven multi-domain workload: Becker tubes (nx ~ U{128..2048} x 4 x 4, shock Mach ~
    U[1.5, 5], Pr 0.75, 8 cells per front, dt-tied omega) and Taylor-Green boxes (N ~ U{32..96},
    M0 ~ U[0.5, 1.25], Re 100), drawn from numpy default_rng(seed)."""
    rng = np.random.default_rng(seed)
    cases = []
    om = becker_tied_omega(8.0)
    for _ in range(n_becker):
        nx = int(rng.integers(128, 2049))
        M = float(rng.uniform(1.5, 5.0))
        cases.append(becker(nx, mach=M, cells_per_front=8.0, omega=om, cfl_max=0.1, ny=4, nz=4,
                            storage=storage))
    for _ in range(n_tgv):
        n = int(rng.integers(32, 97))
        M = float(rng.uniform(0.5, 1.25))
        cases.append(tgv3d(n, mach=M, re=100.0, storage=storage))
    return cases


@dataclass
class Request:
    rid: int
    arrival: float        # seconds after the trace start
    kind: str
    storage: int
    steps: int
    case: Case


def serving_trace(seed: int = 0, n_requests: int = 40, rate: float = 20.0,
                  tgv_range=(64, 192), steps_range=(500, 5000), fp16_prob: float = 0.5):
    """Poisson arrivals (mean `rate` per second) of simulation requests drawn from
    default_rng(seed): type uniform over {Sod tube, Becker tube, Taylor-Green box}, Taylor-Green
    N ~ U{tgv_range}, steps ~ U{steps_range}, FP16 storage with probability fp16_prob (else
    FP32)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    om = becker_tied_omega(8.0)
    for rid in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        kind = ["sod", "becker", "tgv"][int(rng.integers(0, 3))]
        storage = STORE_F16 if rng.uniform() < fp16_prob else STORE_F32
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        if kind == "sod":
            nx = int(rng.integers(400, 4001))
            case = sod(nx, steps=steps, storage=storage, t_end=0.08 * steps / nx)
        elif kind == "becker":
            nx = int(rng.integers(128, 2049))
            case = becker(nx, mach=float(rng.uniform(1.5, 5.0)), cells_per_front=8.0, omega=om,
                          cfl_max=0.1, ny=4, nz=4, storage=storage)
        else:
            n = int(rng.integers(tgv_range[0], tgv_range[1] + 1))
            case = tgv3d(n, mach=float(rng.uniform(0.5, 1.25)), re=100.0, storage=storage)
        reqs.append(Request(rid, t, kind, storage, steps, case))
    return reqs
