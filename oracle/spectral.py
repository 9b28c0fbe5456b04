"""FP64 spectral post-processing of a lattice state (Sec. 3.4): shell-averaged velocity
spectrum and the solenoidal / dilatational dissipation evaluated with spectral derivatives.

TEST INFRASTRUCTURE ONLY: imported by the test suite and the benchmark's CPU legs; never by the
product package.  numpy's FFT is the one library step; everything else is written out here.

Readings of the paper (it states that the dissipation is computed spectrally and shows
shell-averaged spectra, without formulas):
- fields from the lattice-unit conserved moments Q = (rho, m, E) of the state:
  rho_f = max(rho, rho_min), u = m / rho_f, p = max((gamma-1)(E - |m|^2 / (2 rho_f)), p_min),
  T = p / rho_f, mu(T) the collision's closure (constant, or Sutherland
  mu_ref (1 + T_S) t^{3/2} / (t + T_S) with t = T / T_ref);
- u^(m) = sum_x u(x) exp(-2 pi i m.x / n) over the periodic box, m_a in [-n/2, n/2);
- shell b holds the wavevectors with b - 1/2 <= |m| < b + 1/2;
  E(b) = sum over the shell of 1/2 |u^|^2 / N^2, so sum_b E(b) = (1/N) sum_x 1/2 |u|^2;
- d/dx_a <-> i k_a with k_a = 2 pi m_a / n (lattice spacing 1); the Nyquist index
  m_a = -n/2 gets k_a = 0 (the odd derivative of that mode has no real representation);
- eps_s = sum_x mu |curl u|^2, eps_d = sum_x 4/3 mu (div u)^2: lattice-unit volume sums, the
  quantities of the cell-local estimates, with spectral instead of reconstructed gradients.
Only boxes whose extents above 1 are all equal (cubes, or squares with nz = 1) are defined.
"""
from __future__ import annotations

import numpy as np


def _extent(nx, ny, nz):
    ext = [e for e in (nx, ny, nz) if e > 1]
    if not ext or any(e != ext[0] for e in ext):
        raise ValueError("spectral post-processing needs equal extents above 1")
    return ext[0], len(ext)


def shells(nx, ny, nz) -> int:
    """Number of shells: the one of the largest |m| (every component -n/2), plus one."""
    n, d = _extent(nx, ny, nz)
    M = d * (n // 2) ** 2
    return int(np.floor(np.sqrt(M) + 0.5)) + 1


def fields(Q, P):
    """(u (3, N), mu (N,)) from lattice-unit conserved moments Q (5, N) and oracle parameters
    P (lattice units, as built by oracle.lattice_params)."""
    rho_f = np.maximum(Q[0], P.rho_min)
    u = Q[1:4] / rho_f
    p = np.maximum((P.gamma - 1.0) * (Q[4] - 0.5 * (Q[1:4] ** 2).sum(0) / rho_f), P.p_min)
    T = p / rho_f
    mu = np.full(Q.shape[1], P.mu_ref)
    if P.sutherland:
        t = T / P.T_ref
        mu = P.mu_ref * (1.0 + P.T_S) * t ** 1.5 / (t + P.T_S)
    return u, mu


def spectral_diag(u, mu, nx, ny, nz, nbins=None):
    """u (3, N) lattice velocity, mu (N,) lattice viscosity on an nx x ny x nz box (x fastest).
    Returns (E (nbins,), dict(eps_s, eps_d, ke_u)) with the readings of the module docstring."""
    n, _ = _extent(nx, ny, nz)
    N = nx * ny * nz
    nb = shells(nx, ny, nz) if nbins is None else nbins
    shape = (nz, ny, nx)
    uh = [np.fft.fftn(u[a].reshape(shape)) for a in range(3)]
    m = [np.fft.fftfreq(e, d=1.0 / e) if e > 1 else np.zeros(1) for e in (nz, ny, nx)]
    # numpy puts -n/2 at index n/2 (fftfreq), the index of the Nyquist mode
    mz, my, mx = np.meshgrid(*m, indexing="ij")
    M2 = np.rint(mx * mx + my * my + mz * mz).astype(np.int64)
    b = np.floor(np.sqrt(M2) + 0.5).astype(np.int64)
    e = 0.5 * sum(np.abs(h) ** 2 for h in uh) / float(N) ** 2
    E = np.bincount(b.ravel(), weights=e.ravel(), minlength=max(nb, int(b.max()) + 1))[:nb]

    def k_of(mm, ext):
        k = 2.0 * np.pi * mm / ext
        if ext > 1:
            k = np.where(mm == -ext // 2, 0.0, k)
        return k

    kz, ky, kx = k_of(mz, nz), k_of(my, ny), k_of(mx, nx)
    ux, uy, uz = uh
    wx = 1j * (ky * uz - kz * uy)
    wy = 1j * (kz * ux - kx * uz)
    wz = 1j * (kx * uy - ky * ux)
    th = 1j * (kx * ux + ky * uy + kz * uz)
    W = [np.fft.ifftn(h).real.ravel() for h in (wx, wy, wz)]
    TH = np.fft.ifftn(th).real.ravel()
    eps_s = float((mu * (W[0] ** 2 + W[1] ** 2 + W[2] ** 2)).sum())
    eps_d = float((4.0 / 3.0 * mu * TH ** 2).sum())
    ke_u = float(0.5 * (u * u).sum())
    return E, dict(eps_s=eps_s, eps_d=eps_d, ke_u=ke_u)


def from_oracle(orc, nbins=None):
    """Spectral diagnostics of an Oracle's current state."""
    u, mu = fields(orc.conserved_lattice(), orc.P)
    return spectral_diag(u, mu, orc.prm.nx, orc.prm.ny, orc.prm.nz, nbins)
