"""FP64 CPU oracle of the five-field gradient-reconstruction LBM (arxiv 2609.16361).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the CPU-baseline
leg of the benchmark; never by the product package.  It shares no code with the CUDA path.

`Oracle` wraps the C stepper in `grlb_oracle.c` (compiled here with gcc + OpenMP) and does its
own conversion of a physical-unit case to lattice units (dx = dt = 1):
  rho unchanged; u_L = s u; p_L, E_L, T_L = s^2 (p, E, T); mu_L = mu dt/dx^2, same for kappa;
  with s = dt/dx.  kappa = mu c_p / Pr with c_p = gamma/(gamma - 1) (T = p/rho, R = 1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grlb_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libgrlb_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc -O2 -fopenmp)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("bc", C.c_int),
                ("collision", C.c_int), ("sutherland", C.c_int), ("gamma", C.c_double),
                ("mu_ref", C.c_double), ("kappa_ref", C.c_double), ("T_ref", C.c_double),
                ("T_S", C.c_double), ("omega", C.c_double * 5), ("omega_min", C.c_double),
                ("gain", C.c_double), ("J_min", C.c_double), ("rho_min", C.c_double),
                ("p_min", C.c_double), ("left", C.c_double * 5), ("right", C.c_double * 5)]


class CellInfo(C.Structure):
    _fields_ = [("Q", C.c_double * 5), ("rho", C.c_double), ("u", C.c_double * 3),
                ("p", C.c_double), ("T", C.c_double), ("mu", C.c_double),
                ("kappa", C.c_double), ("gradQ", C.c_double * 15), ("gradu", C.c_double * 9),
                ("gradT", C.c_double * 3), ("chi", C.c_double), ("floored", C.c_int)]


CELL_DTYPE = np.dtype([("Q", "f8", 5), ("rho", "f8"), ("u", "f8", 3), ("p", "f8"),
                       ("T", "f8"), ("mu", "f8"), ("kappa", "f8"), ("gradQ", "f8", 15),
                       ("gradu", "f8", 9), ("gradT", "f8", 3), ("chi", "f8"),
                       ("floored", "i4"), ("_pad", "i4")])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            L.orc_step.argtypes = [C.POINTER(_Params), dp, dp, C.c_void_p]
            L.orc_step.restype = C.c_int
            L.orc_step_src.argtypes = [C.POINTER(_Params), dp, dp, C.c_void_p, C.c_void_p]
            L.orc_step_src.restype = C.c_int
            L.orc_cell.argtypes = [C.POINTER(_Params), dp, dp, C.POINTER(CellInfo)]
            L.orc_cell.restype = C.c_int
            L.orc_init_equilibrium.argtypes = [C.POINTER(_Params), dp, dp, dp, dp, dp, dp]
            L.orc_init_equilibrium.restype = None
            L.orc_equilibrium_state.argtypes = [C.POINTER(_Params), dp, dp]
            L.orc_equilibrium_state.restype = None
            L.orc_moments.argtypes = [C.POINTER(_Params), dp, dp]
            L.orc_moments.restype = None
            L.orc_cell_info_size.restype = C.c_size_t
            L.orc_num_threads.restype = C.c_int
            assert L.orc_cell_info_size() == CELL_DTYPE.itemsize == C.sizeof(CellInfo)
            _lib = L
        return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lattice_params(prm) -> _Params:
    """Physical-unit CaseParams -> lattice-unit oracle parameters."""
    s = prm.dt / prm.dx
    g = prm.gamma
    cp = g / (g - 1.0)
    mu_L = prm.mu_ref * prm.dt / prm.dx ** 2
    kap_L = mu_L * cp / prm.prandtl
    P = _Params()
    P.nx, P.ny, P.nz = prm.nx, prm.ny, prm.nz
    P.bc, P.collision, P.sutherland = prm.bc, prm.collision, prm.sutherland
    P.gamma = g
    P.mu_ref, P.kappa_ref = mu_L, kap_L
    P.T_ref = prm.T_ref * s * s
    P.T_S = prm.T_S
    om = [prm.omega_rho, prm.omega_mom, prm.omega_mom, prm.omega_mom, prm.omega_E]
    for k in range(5):
        P.omega[k] = om[k]
    P.omega_min, P.gain, P.J_min = prm.omega_min, prm.sensor_gain, prm.J_min
    P.rho_min, P.p_min = prm.rho_min, prm.p_min * s * s

    def prim_L(pr):
        return (pr[0], pr[1] * s, pr[2] * s, pr[3] * s, pr[4] * s * s)

    for k, v in enumerate(prim_L(prm.left_prim)):
        P.left[k] = v
    for k, v in enumerate(prim_L(prm.right_prim)):
        P.right[k] = v
    return P


class Oracle:
    """FP64 stepper for one domain of a physical-unit case."""

    def __init__(self, prm):
        self.prm = prm
        self.P = lattice_params(prm)
        self.s = prm.dt / prm.dx
        self.N = prm.nx * prm.ny * prm.nz
        self.f = np.zeros((35, self.N))
        self.g = np.zeros((35, self.N))
        self.steps = 0
        self.last_cells = None

    # -- state --------------------------------------------------------------------------
    def init_primitive(self, rho, u, p, ce_init: bool = False):
        """Populations of the physical primitive fields: the equilibrium f^eq(Q, Phi^adv), plus
        with ce_init the Chapman-Enskog non-equilibrium part (chapman_enskog_moments)."""
        s = self.s
        rho = np.ascontiguousarray(rho, np.float64)
        ux = np.ascontiguousarray(u[0] * s)
        uy = np.ascontiguousarray(u[1] * s)
        uz = np.ascontiguousarray(u[2] * s)
        pL = np.ascontiguousarray(np.asarray(p, np.float64) * s * s)
        lib().orc_init_equilibrium(C.byref(self.P), _dp(rho), _dp(ux), _dp(uy), _dp(uz),
                                   _dp(pL), _dp(self.f))
        if ce_init:
            A = self.chapman_enskog_moments(rho, u, p)
            # w_i c_i . A_k / cs^2 with w_i / cs^2 = 1/2 on the six links
            for k in range(5):
                for a in range(3):
                    self.f[7 * k + 1 + 2 * a] += 0.5 * A[k, a]
                    self.f[7 * k + 2 + 2 * a] -= 0.5 * A[k, a]
        self.steps = 0

    def chapman_enskog_moments(self, rho, u, p):
        """Non-equilibrium first moments A_k (5, 3, N), lattice units, of the Chapman-Enskog
        state the first sweep streams (Sec. 2.3: the non-equilibrium first moment of field k
        carries its gradient).  Before the collision the streamed first moment is
        J_k = Phi^adv_k + Phi^diff_k - tau_k cs^2 grad Q_k; after the collision (regularized
        or BGK, nominal tau_k = 1/omega_k) the stored populations carry
        A_k = Phi^diff_k - (tau_k - 1) cs^2 grad Q_k on top of f^eq(Q, Phi^adv).
        Gradients: central differences (phi(x + e_a) - phi(x - e_a)) / 2 of Q_k, u and T,
        periodic, or with the ghost states beyond the ends of an X_DIRICHLET_EQ tube; zero
        along an axis of extent 1.  Phi^diff: 0 (rho), -tau_visc (momentum),
        -tau_visc u + q (energy); tau_visc = mu (grad u + grad u^T - 2/3 div u I),
        q = -kappa grad T, mu and kappa at the local T (constant or Sutherland)."""
        P, s, prm = self.P, self.s, self.prm
        nx, ny, nz = prm.nx, prm.ny, prm.nz
        g = prm.gamma
        rho = np.asarray(rho, np.float64)
        uL = np.asarray(u, np.float64) * s
        pL = np.asarray(p, np.float64) * s * s
        T = pL / rho
        Q = np.stack([rho, rho * uL[0], rho * uL[1], rho * uL[2],
                      pL / (g - 1.0) + 0.5 * rho * (uL * uL).sum(0)])

        def ghost(prim):
            r, gx, gy, gz, gp = prim[0], prim[1] * s, prim[2] * s, prim[3] * s, prim[4] * s * s
            return dict(Q=[r, r * gx, r * gy, r * gz, gp / (g - 1.0) + 0.5 * r * (gx * gx + gy * gy + gz * gz)],
                        u=[gx, gy, gz], T=gp / r)

        gl, gr = ghost(prm.left_prim), ghost(prm.right_prim)

        def grad(phi, left, right):
            a = phi.reshape(nz, ny, nx)
            out = np.zeros((3,) + a.shape)
            if nx > 1:
                if prm.bc == 1:
                    pad = np.concatenate([np.full((nz, ny, 1), left), a, np.full((nz, ny, 1), right)], axis=2)
                    out[0] = 0.5 * (pad[:, :, 2:] - pad[:, :, :-2])
                else:
                    out[0] = 0.5 * (np.roll(a, -1, axis=2) - np.roll(a, 1, axis=2))
            if ny > 1:
                out[1] = 0.5 * (np.roll(a, -1, axis=1) - np.roll(a, 1, axis=1))
            if nz > 1:
                out[2] = 0.5 * (np.roll(a, -1, axis=0) - np.roll(a, 1, axis=0))
            return out.reshape(3, -1)

        gQ = np.stack([grad(Q[k], gl["Q"][k], gr["Q"][k]) for k in range(5)])   # [k, a]
        gu = np.stack([grad(uL[j], gl["u"][j], gr["u"][j]) for j in range(3)])  # [j, a] = d_a u_j
        gT = grad(T, gl["T"], gr["T"])
        fac = np.ones_like(T)
        if P.sutherland:
            t = T / P.T_ref
            fac = (1.0 + P.T_S) * t ** 1.5 / (t + P.T_S)
        mu, kap = P.mu_ref * fac, P.kappa_ref * fac
        th = gu[0, 0] + gu[1, 1] + gu[2, 2]
        tv = np.empty((3, 3) + T.shape)
        for j in range(3):
            for a in range(3):
                tv[j, a] = mu * (gu[j, a] + gu[a, j] - (2.0 / 3.0 * th if j == a else 0.0))
        q = -kap * gT
        diff = np.zeros((5, 3) + T.shape)
        for j in range(3):
            diff[1 + j] = -tv[j]
        for a in range(3):
            diff[4, a] = -(tv[a, 0] * uL[0] + tv[a, 1] * uL[1] + tv[a, 2] * uL[2]) + q[a]
        tau = 1.0 / np.array([P.omega[0], P.omega[1], P.omega[2], P.omega[3], P.omega[4]])
        return diff - ((tau - 1.0) * 0.25)[:, None, None] * gQ

    def source_lattice(self, S):
        """Physical source rates (5, N) -> lattice units per step: rho dt, m dt s, E dt s^2."""
        s, dt = self.s, self.prm.dt
        out = np.array(S, dtype=np.float64, copy=True)
        out[0] *= dt
        out[1:4] *= dt * s
        out[4] *= dt * s * s
        return np.ascontiguousarray(out)

    def step(self, n: int = 1, keep_cells: bool = False, source=None):
        """Advance n steps.  source(step) -> physical source rates (5, N) applied in that step
        (projected as w_i S_k after the collision, Alg. 1 step 9), or None."""
        L = lib()
        for it in range(n):
            cells = None
            if keep_cells and it == n - 1:
                cells = np.zeros(self.N, CELL_DTYPE)
            S = None if source is None else self.source_lattice(source(self.steps))
            rc = L.orc_step_src(C.byref(self.P), _dp(self.f), _dp(self.g),
                                None if cells is None else cells.ctypes.data_as(C.c_void_p),
                                None if S is None else S.ctypes.data_as(C.c_void_p))
            if rc != 0:
                raise RuntimeError("oracle: singular reconstruction system")
            self.f, self.g = self.g, self.f
            self.steps += 1
            if cells is not None:
                self.last_cells = cells

    # -- readback (physical units) -------------------------------------------------------
    def conserved_lattice(self):
        Q = np.zeros((5, self.N))
        lib().orc_moments(C.byref(self.P), _dp(self.f), _dp(Q))
        return Q

    def conserved(self):
        """(rho, m_x, m_y, m_z, E) in physical units, shape (5, N)."""
        Q = self.conserved_lattice()
        s = self.s
        Q[1:4] /= s
        Q[4] /= s * s
        return Q

    def primitive(self):
        """rho, u (3, N), p, T in physical units (no floors)."""
        Q = self.conserved()
        rho = Q[0]
        u = Q[1:4] / rho
        p = (self.prm.gamma - 1.0) * (Q[4] - 0.5 * rho * (u * u).sum(0))
        return rho, u, p, p / rho

    def diagnostics_from_cells(self, cells=None):
        """Lattice-unit volume sums of the state the last step landed on (pre-collision):
        totals of Q_k, kinetic energy 1/2|m|^2/rho, solenoidal mu|curl u|^2 and dilatational
        (4/3) mu (div u)^2 dissipation, min rho, min p, floor hits, sensor hits."""
        c = self.last_cells if cells is None else cells
        gu = c["gradu"].reshape(-1, 3, 3)
        wx = gu[:, 2, 1] - gu[:, 1, 2]
        wy = gu[:, 0, 2] - gu[:, 2, 0]
        wz = gu[:, 1, 0] - gu[:, 0, 1]
        th = gu[:, 0, 0] + gu[:, 1, 1] + gu[:, 2, 2]
        m = c["Q"][:, 1:4]
        return dict(totals=c["Q"].sum(0),
                    ke=float((0.5 * (m * m).sum(1) / c["rho"]).sum()),
                    eps_s=float((c["mu"] * (wx * wx + wy * wy + wz * wz)).sum()),
                    eps_d=float((4.0 / 3.0 * c["mu"] * th * th).sum()),
                    rho_min=float(c["rho"].min()), p_min=float(c["p"].min()),
                    n_floor=int(c["floored"].sum()), n_sensor=int((c["chi"] > 0).sum()))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def cell(P: _Params, fhat: np.ndarray):
    """Run Algorithm 1 on one cell; returns (fstar[35], CellInfo)."""
    fhat = np.ascontiguousarray(fhat, np.float64)
    out = np.zeros(35)
    info = CellInfo()
    rc = lib().orc_cell(C.byref(P), _dp(fhat), _dp(out), C.byref(info))
    if rc != 0:
        raise RuntimeError("oracle: singular reconstruction system")
    return out, info


def equilibrium_state(P: _Params, prim) -> np.ndarray:
    out = np.zeros(35)
    pr = np.ascontiguousarray(prim, np.float64)
    lib().orc_equilibrium_state(C.byref(P), _dp(pr), _dp(out))
    return out
