"""Pins of the oracle's spectral post-processing (Sec. 3.4: spectrally computed dissipation,
shell-averaged velocity spectrum).

Expected values are closed forms of single Fourier modes (energy in one shell, |curl u|^2 and
(div u)^2 of a sine), Parseval's identity, the Taylor-Green initial field (all energy at
|m| = sqrt 3, mean |curl u|^2 = 3/4 V0^2/L0^2, zero divergence), and the second-order agreement
of the collision's reconstructed gradients with spectral ones.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import spectral
from paper_2609_16361_b300 import inputs


def grid(n, nz=None):
    nz = n if nz is None else nz
    z, y, x = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def test_shell_count():
    assert spectral.shells(16, 16, 16) == int(math.floor(math.sqrt(3) * 8 + 0.5)) + 1  # 15
    assert spectral.shells(16, 16, 1) == 12  # sqrt(2) 8 = 11.31 -> shell 11
    with pytest.raises(ValueError):
        spectral.shells(16, 8, 8)


@pytest.mark.parametrize("m0", [1, 3, 7])
def test_shear_mode(m0):
    n, A, mu = 16, 0.02, 0.003
    x, y, z = grid(n)
    k0 = 2 * math.pi * m0 / n
    u = np.zeros((3, n ** 3))
    u[0] = A * np.sin(k0 * y)
    E, s = spectral.spectral_diag(u, np.full(n ** 3, mu), n, n, n)
    # 1/2 <u^2> = A^2/4, all in shell m0
    assert E[m0] == pytest.approx(A * A / 4, rel=1e-12)
    assert np.abs(np.delete(E, m0)).max() < 1e-15 * A * A
    # curl u = (0, 0, -A k0 cos k0 y): sum mu |omega|^2 = N mu A^2 k0^2 / 2
    assert s["eps_s"] == pytest.approx(n ** 3 * mu * A * A * k0 * k0 / 2, rel=1e-12)
    assert s["eps_d"] < 1e-12 * s["eps_s"]


def test_compressive_mode():
    n, A, mu = 16, 0.02, 0.003
    x, y, z = grid(n)
    k0 = 2 * math.pi * 2 / n
    u = np.zeros((3, n ** 3))
    u[0] = A * np.sin(k0 * x)
    E, s = spectral.spectral_diag(u, np.full(n ** 3, mu), n, n, n)
    # div u = A k0 cos k0 x: sum 4/3 mu theta^2 = 4/3 N mu A^2 k0^2 / 2
    assert s["eps_d"] == pytest.approx(4.0 / 3.0 * n ** 3 * mu * A * A * k0 * k0 / 2, rel=1e-12)
    assert s["eps_s"] < 1e-12 * s["eps_d"]
    assert E[2] == pytest.approx(A * A / 4, rel=1e-12)


def test_oblique_mode_shell_and_curl():
    """u_z = A cos(2 pi (2x + 3y)/n): |m| = sqrt 13 = 3.61 lies in shell 4."""
    n, A, mu = 16, 0.01, 0.002
    x, y, z = grid(n)
    k1, k2 = 2 * math.pi * 2 / n, 2 * math.pi * 3 / n
    u = np.zeros((3, n ** 3))
    u[2] = A * np.cos(k1 * x + k2 * y)
    E, s = spectral.spectral_diag(u, np.full(n ** 3, mu), n, n, n)
    assert E[4] == pytest.approx(A * A / 4, rel=1e-12)
    assert E[3] < 1e-15 and E[5] < 1e-15
    # curl u = (d_y u_z, -d_x u_z, 0): |omega|^2 = A^2 (k1^2 + k2^2) sin^2
    assert s["eps_s"] == pytest.approx(n ** 3 * mu * A * A * (k1 * k1 + k2 * k2) / 2, rel=1e-12)


def test_nyquist_mode_has_no_derivative():
    """Reading: the Nyquist index contributes energy to shell n/2 but no derivative."""
    n, A = 16, 0.01
    x, y, z = grid(n)
    u = np.zeros((3, n ** 3))
    u[1] = A * (-1.0) ** x
    E, s = spectral.spectral_diag(u, np.full(n ** 3, 1e-3), n, n, n)
    assert E[n // 2] == pytest.approx(A * A / 2, rel=1e-12)
    assert s["eps_s"] < 1e-25 and s["eps_d"] < 1e-25


def test_parseval_random_field():
    rng = np.random.default_rng(5)
    n = 16
    u = rng.normal(size=(3, n ** 3)) * 0.01
    E, s = spectral.spectral_diag(u, np.full(n ** 3, 1e-3), n, n, n)
    assert E.sum() == pytest.approx(s["ke_u"] / n ** 3, rel=1e-12)
    assert s["ke_u"] == pytest.approx(0.5 * (u * u).sum(), rel=1e-14)


def test_square_2d_box():
    n, A, mu = 32, 0.02, 0.004
    x, y, z = grid(n, nz=1)
    k0 = 2 * math.pi * 5 / n
    u = np.zeros((3, n * n))
    u[0] = A * np.cos(k0 * y)
    E, s = spectral.spectral_diag(u, np.full(n * n, mu), n, n, 1)
    assert len(E) == spectral.shells(n, n, 1)
    assert E[5] == pytest.approx(A * A / 4, rel=1e-12)
    assert s["eps_s"] == pytest.approx(n * n * mu * A * A * k0 * k0 / 2, rel=1e-12)


def test_fields_floors_and_sutherland():
    P = oracle.lattice_params(inputs.uniform(4, 1, 1, sutherland=1).params.replace(
        dx=1.0, dt=1.0, mu_ref=0.01, T_ref=0.5, T_S=0.5, rho_min=0.1, p_min=1e-3, gamma=1.4))
    # rho below the floor: u = m / rho_min; T = T_ref gives mu = mu_ref exactly;
    # T = 4 T_ref gives mu_ref (1 + 1/2) 8 / (4 + 1/2) = 8/3 mu_ref
    rho = np.array([0.05, 1.0, 1.0])
    m = np.array([[0.01, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    p = np.array([0.05, 0.5, 2.0])  # T = p / rho_f = 0.5, 0.5, 2.0
    E = p / 0.4 + 0.5 * (m * m).sum(0) / np.maximum(rho, 0.1)
    Q = np.stack([rho, m[0], m[1], m[2], E])
    u, mu = spectral.fields(Q, P)
    assert u[0, 0] == pytest.approx(0.01 / 0.1, rel=1e-14)
    assert mu[0] == pytest.approx(0.01, rel=1e-12)   # T = 0.05/0.1 = T_ref
    assert mu[1] == pytest.approx(0.01, rel=1e-12)
    assert mu[2] == pytest.approx(0.01 * 8.0 / 3.0, rel=1e-12)


def tgv_closed_form(case):
    """Taylor-Green initial field, lattice units: E in shell 2 (|m| = sqrt 3) equals
    1/2 <|u_L|^2> = s^2 / 8; sum mu |curl u_L|^2 = N mu_L (s dx)^2 3/4; div u = 0."""
    s, dx, n = case.params.dt / case.params.dx, case.params.dx, case.params.nx
    return s * s / 8.0, n ** 3 * (s * dx) ** 2 * 0.75


@pytest.mark.parametrize("n", [16, 32])
def test_taylor_green_initial_field(n):
    c = inputs.tgv3d(n, mach=0.5, re=100.0)
    o = oracle.Oracle(c.params)
    o.init_primitive(c.rho, c.u, c.p)
    E, s = spectral.from_oracle(o)
    e2, eps_per_mu = tgv_closed_form(c)
    assert E[2] == pytest.approx(e2, rel=1e-12)
    assert E.sum() == pytest.approx(e2, rel=1e-12)
    # uniform T = T_ref at t = 0, so Sutherland's mu is mu_ref
    assert s["eps_s"] == pytest.approx(o.P.mu_ref * eps_per_mu, rel=1e-10)
    assert s["eps_d"] < 1e-20 * s["eps_s"] + 1e-30


def test_reconstructed_dissipation_converges_to_spectral():
    """The collision's cell-local eps_s (gradients reconstructed from the non-equilibrium
    moments, Eq. gradrecon) approaches the spectral eps_s at second order on a smooth,
    viscous Taylor-Green flow (Re 20, M 0.3): error 3.6 % at 16^3, 0.7 % at 32^3."""
    errs = []
    for n in (16, 32):
        c = inputs.tgv3d(n, mach=0.3, re=20.0, sutherland=0, fmu=1.0)
        o = oracle.Oracle(c.params)
        o.init_primitive(c.rho, c.u, c.p)
        o.step(24)
        o.step(1, keep_cells=True)
        cell = o.diagnostics_from_cells()["eps_s"]
        _, s = spectral.from_oracle(o)
        errs.append(abs(cell / s["eps_s"] - 1.0))
    assert errs[0] < 0.05 and errs[1] < 0.012
    assert math.log2(errs[0] / errs[1]) > 1.8
