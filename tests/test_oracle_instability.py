"""The finding that the regularized collision with the linear equilibrium is unstable near
omega = 2, pinned twice:

- on the scalar model the finding is derived from (one advected field on the 1-D reduction of
  D3Q7: rest weight 3/4, link weights 1/8, cs^2 = 1/4, equilibrium w_i (Q + c_i a Q / cs^2)),
  built here from those definitions alone: at omega = 2 the regularized map (Q, J) ->
  (Q, omega a Q + (1 - omega) J) followed by streaming has, at cos k = -1/3, an eigenvalue of
  modulus sqrt(1 + 4 a^2 sin^2 k) > 1 for every a != 0, whereas BGK at omega = 2 keeps every
  eigenvalue on or inside the unit circle up to |a| = 1/4 and leaves it beyond;
- on the FP64 oracle (five fields, full Euler flux): a 1e-10 pressure perturbation of a
  uniform moving state whose characteristic speeds stay below 1/4 (|u| + c = 0.17 in lattice
  units) grows by more than 1e3 over 180 steps under the regularized collision at omega = 1.99
  and stays bounded under BGK.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2609_16361_b300 import inputs

W = np.array([0.75, 0.125, 0.125])
C = np.array([0.0, 1.0, -1.0])
CS2 = 0.25


def stream(k):
    return np.diag(np.exp(-1j * C * k))  # f_i(x) <- f*_i(x - c_i)


def rlb_map(a, omega):
    Jstar = omega * a * np.ones(3) + (1.0 - omega) * C
    return np.outer(W, np.ones(3)) + np.outer(W * C / CS2, Jstar)


def bgk_map(a, omega):
    E = np.outer(W * (1.0 + C * a / CS2), np.ones(3))
    return np.eye(3) + omega * (E - np.eye(3))


def spectral_radius(M, k):
    return np.abs(np.linalg.eigvals(stream(k) @ M)).max()


@pytest.mark.parametrize("a", [0.02, 0.05, 0.1, 0.2])
def test_regularized_eigenvalue_closed_form(a):
    k = math.acos(-1.0 / 3.0)
    assert spectral_radius(rlb_map(a, 2.0), k) == pytest.approx(math.sqrt(1 + 4 * a * a * math.sin(k) ** 2),
                                                                rel=1e-12)


def test_bgk_at_omega_two_is_stable_up_to_a_quarter():
    ks = np.linspace(1e-3, math.pi, 1201)
    for a in (0.05, 0.1, 0.2, 0.25):
        assert max(spectral_radius(bgk_map(a, 2.0), k) for k in ks) <= 1 + 1e-9, a
    assert max(spectral_radius(bgk_map(0.27, 2.0), k) for k in ks) > 1 + 1e-3
    assert max(spectral_radius(rlb_map(0.05, 2.0), k) for k in ks) > 1 + 1e-3


def perturbation_growth(collision, steps=180):
    c = inputs.uniform(64, 1, 1, u=(0.1, 0.0, 0.0), p=0.04114, collision=collision)
    prm = c.params.replace(omega_rho=1.99, omega_mom=1.99, omega_E=1.99, sensor_gain=0.0, mu_ref=1e-6)
    x = np.arange(64)
    p = c.p * (1 + 1e-10 * np.sin(2 * np.pi * 21 * x / 64))
    o = oracle.Oracle(prm)
    o.init_primitive(c.rho, c.u, p)
    o.step(20)  # the pressure perturbation has reached the density by now
    a0 = np.abs(o.conserved()[0] - c.rho[0]).max()
    o.step(steps)
    return np.abs(o.conserved()[0] - c.rho[0]).max() / a0


def test_oracle_regularized_grows_bgk_stays_bounded():
    assert perturbation_growth(inputs.COLL_RLB_SENSOR) > 1e3
    assert perturbation_growth(inputs.COLL_BGK) < 2.0
