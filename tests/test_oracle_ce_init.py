"""Pins of the oracle's Chapman-Enskog initialisation (Sec. 2.3: the non-equilibrium first
moment of a field carries its gradient).

The state it writes is the post-collision state of a smooth flow, so the gradients that the
collision reconstructs from the streamed populations match the spectral gradients of the field
from the first step on, at omega near 2 as well; the equilibrium start instead leaves a
non-equilibrium part that flips sign every step (the reconstructed dissipation alternates
between about 4x and 0x its value).  A wrong sign, or tau instead of tau - 1 in the stored
non-equilibrium moment, brings the alternation back.  A uniform field has no gradient, so the
start is the equilibrium one; the conserved moments never change.
"""
import numpy as np
import pytest

import oracle
from oracle import spectral
from paper_2609_16361_b300 import inputs


def start(case, ce):
    o = oracle.Oracle(case.params)
    o.init_primitive(case.rho, case.u, case.p, ce_init=ce)
    return o


def dissipation_ratio(o, steps):
    out = []
    for _ in range(steps):
        o.step(1, keep_cells=True)
        cell = o.diagnostics_from_cells()["eps_s"]
        _, sp = spectral.from_oracle(o)
        out.append(cell / sp["eps_s"])
    return np.array(out)


@pytest.mark.parametrize("fmu", [0.001, 1.0])
def test_reconstructed_dissipation_without_alternation(fmu):
    c = inputs.tgv3d(32, mach=0.5, re=100.0, sutherland=0, fmu=fmu)
    r_ce = dissipation_ratio(start(c, True), 4)
    r_eq = dissipation_ratio(start(c, False), 4)
    assert np.all(np.abs(r_ce - 1.0) < 0.03), r_ce
    assert r_eq[0] > 2.5 and r_eq[1] < 0.1 and r_eq[2] > 2.5 and r_eq[3] < 0.2, r_eq


def test_uniform_field_is_the_equilibrium_start():
    c = inputs.uniform(8, 6, 4)
    assert np.array_equal(start(c, True).f, start(c, False).f)


def test_conserved_moments_unchanged():
    c = inputs.random_smooth(12, 10, 8, seed=7)
    a, b = start(c, True), start(c, False)
    assert np.abs(a.f - b.f).max() > 1e-6
    np.testing.assert_allclose(a.conserved_lattice(), b.conserved_lattice(), rtol=0, atol=1e-14)


def test_tube_ends_use_the_ghost_states():
    """Sod: the ghost states equal the adjacent end states, so the ends carry no gradient and
    no non-equilibrium part (a periodic wrap would see the full jump there)."""
    c = inputs.sod(64)
    o = oracle.Oracle(c.params)
    A = o.chapman_enskog_moments(c.rho, c.u, c.p)
    nx = c.params.nx
    assert np.abs(A[:, :, 0]).max() == 0.0 and np.abs(A[:, :, nx - 1]).max() == 0.0
    assert np.abs(A[:, 0, nx // 2]).max() > 1e-3
