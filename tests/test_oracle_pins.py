"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics.

Nothing here compares the oracle with itself: every expected value is a closed form
(Euler flux, Newtonian stress / Fourier flux from their definitions, exact Riemann and Becker
solutions, incompressible Taylor-Green decay), an invariant (conservation, uniform state), or
a number the paper prints (its convergence tables, beta at the Taylor-Green point).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2609_16361_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CI = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
WI = np.array([0.25] + [0.125] * 6)
CS2 = 0.25


def lattice_P(**kw):
    base = inputs.uniform(4, 1, 1, sutherland=0).params.replace(dx=1.0, dt=1.0)
    return oracle.lattice_params(base.replace(**kw))


def pops_with_moments(Q, J):
    """Any population set with zeroth moments Q[5] and first moments J[5,3]."""
    f = np.zeros(35)
    for k in range(5):
        for i in range(7):
            f[7 * k + i] = WI[i] * (Q[k] + CI[i] @ J[k] / CS2)
    return f


def euler_flux(rho, u, p, gamma):
    m = rho * u
    E = p / (gamma - 1) + 0.5 * rho * u @ u
    F = np.zeros((5, 3))
    F[0] = m
    F[1:4] = np.outer(m, u) + p * np.eye(3)
    F[4] = (E + p) * u
    return np.array([rho, *m, E]), F


# ---- equilibrium --------------------------------------------------------------------------
def test_equilibrium_moments_are_state_and_euler_flux():
    rng = np.random.default_rng(3)
    P = lattice_P()
    for _ in range(10):
        rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.1, 1.0)
        u = rng.uniform(-0.2, 0.2, 3)
        f = oracle.equilibrium_state(P, [rho, *u, p]).reshape(5, 7)
        Q, F = euler_flux(rho, u, p, 1.4)
        np.testing.assert_allclose(f.sum(1), Q, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(f @ CI, F, rtol=1e-13, atol=1e-15)
        # second moment of the linear equilibrium is cs^2 Q I with cs^2 = 1/4 (Sec. 2.2)
        for k in range(5):
            M2 = np.einsum("i,ia,ib->ab", f[k], CI, CI)
            np.testing.assert_allclose(M2, CS2 * Q[k] * np.eye(3), atol=1e-14)


# ---- reconstruction operator (Eqs. gradrecon, feedback, cnsfM, cnsfE) ---------------------
def build_first_moments(rho, u, p, gr, gu, gT, mu, kappa, omega, gamma):
    """First moments a Chapman-Enskog-consistent population set carries: J = Phi^adv +
    Phi^diff - cs^2 tau_LB grad Q, with Phi^diff from the Newtonian stress and Fourier flux
    definitions (Eq. system), NOT from the Jacobian M."""
    T = p / rho
    gp = T * gr + rho * gT
    gm = rho * gu + np.outer(u, gr)                 # (grad m)_{jc}
    gE = gp / (gamma - 1) + 0.5 * (u @ u) * gr + rho * (gu.T @ u)
    gradQ = np.vstack([gr, gm, gE])                 # (5, 3)
    Q, Fadv = euler_flux(rho, u, p, gamma)
    div = np.trace(gu)
    tau = mu * (gu + gu.T - 2.0 / 3.0 * div * np.eye(3))
    q = -kappa * gT
    Fdiff = np.zeros((5, 3))
    Fdiff[1:4] = -tau
    Fdiff[4] = -tau @ u + q
    J = Fadv + Fdiff - CS2 / np.asarray(omega)[:, None] * gradQ
    return Q, J, gradQ


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("sutherland", [0, 1])
def test_reconstruction_recovers_exact_gradients(seed, sutherland):
    rng = np.random.default_rng(seed)
    g = 1.4
    rho, p = rng.uniform(0.6, 1.8), rng.uniform(0.05, 0.5)
    u = rng.uniform(-0.15, 0.15, 3)
    mu_ref = rng.uniform(0.0, 0.4)
    pr = rng.uniform(0.5, 1.0)
    om = rng.uniform(1.2, 2.0, 3)
    omega = np.array([om[0], om[1], om[1], om[1], om[2]])
    T_ref = rng.uniform(0.1, 0.5)
    P = lattice_P(gamma=g, mu_ref=mu_ref, prandtl=pr, T_ref=T_ref, sutherland=sutherland,
                  omega_rho=om[0], omega_mom=om[1], omega_E=om[2], collision=0)
    T = p / rho
    if sutherland:
        t = T / T_ref
        mu = mu_ref * (1 + 0.4042) * t ** 1.5 / (t + 0.4042)   # Listing 1
    else:
        mu = mu_ref
    kappa = mu * (g / (g - 1)) / pr
    gr = rng.normal(0, 0.05, 3)
    gu = rng.normal(0, 0.05, (3, 3))
    gT = rng.normal(0, 0.01, 3)
    Q, J, gradQ = build_first_moments(rho, u, p, gr, gu, gT, mu, kappa, omega, g)
    _, info = oracle.cell(P, pops_with_moments(Q, J))
    np.testing.assert_allclose(np.array(info.gradQ).reshape(5, 3), gradQ, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(np.array(info.gradu).reshape(3, 3), gu, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(np.array(info.gradT), gT, rtol=1e-9, atol=1e-12)
    assert info.mu == pytest.approx(mu, rel=1e-13)
    assert info.kappa == pytest.approx(kappa, rel=1e-13)


def test_momentum_block_damps_only_symmetric_deviatoric_part_by_one_plus_beta():
    """Sec. 2.4: vorticity and dilatation pass undamped, sym-dev strain scaled by
    1/(1+beta), beta = 2 nu omega / cs^2 (Eq. beta).  State at rest, no density gradient."""
    rho, p, mu, om = 1.3, 0.3, 0.05, 1.7
    P = lattice_P(mu_ref=mu, prandtl=1e30, omega_rho=om, omega_mom=om, omega_E=om, collision=0)
    beta = 2 * (mu / rho) * om / CS2
    G = np.array([[0.01, 0.03, -0.02], [0.005, -0.04, 0.01], [0.02, 0.0, 0.015]])
    Q = np.array([rho, 0, 0, 0, p / 0.4])
    J = np.zeros((5, 3))
    J[1:4] = p * np.eye(3) - CS2 / om * G       # g~_m = G exactly
    _, info = oracle.cell(P, pops_with_moments(Q, J))
    gm = np.array(info.gradQ).reshape(5, 3)[1:4]
    sym = 0.5 * (G + G.T)
    dev = sym - np.trace(G) / 3 * np.eye(3)
    expect = G - dev + dev / (1 + beta)
    np.testing.assert_allclose(gm, expect, rtol=1e-12, atol=1e-15)


def test_beta_at_taylor_green_point_matches_paper():
    """beta ~ 0.02 at the compressible Taylor-Green point (Sec. 2.4), here at 128^3 with
    dt = 0.1 dx on the 2 pi box; beta grows linearly with N under acoustic scaling."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))["beta_ctgv"]["value"]
    c = inputs.tgv3d(128, nxyz=(4, 4, 4))
    P = oracle.lattice_params(c.params)
    beta = 2 * (P.mu_ref / 1.0) * P.omega[1] / CS2
    assert beta == pytest.approx(gold, rel=0.1)


# ---- floors and sensor (Alg. 1, Listing 2) -----------------------------------------------
def test_positivity_floors():
    P = lattice_P(rho_min=1e-4, p_min=1e-4, collision=1)
    Q = np.array([1.0, 0.1, 0.0, 0.0, 0.001])     # E below kinetic energy -> p < 0
    _, info = oracle.cell(P, pops_with_moments(Q, np.zeros((5, 3))))
    assert info.floored == 1 and info.p == pytest.approx(P.p_min)
    Q = np.array([1e-6, 0.0, 0.0, 0.0, 1.0])
    _, info = oracle.cell(P, pops_with_moments(Q, np.zeros((5, 3))))
    assert info.floored == 1 and info.rho == pytest.approx(1e-4)


def test_sensor_gate_uniform_compression():
    """chi = clamp(g s, 0, 1) with s = -div u / cs, only in compression above J_min."""
    g, jmin = 20.0, 3e-3
    P = lattice_P(mu_ref=0.0, sensor_gain=g, J_min=jmin, collision=1)
    rho, p, u = 1.0, 0.5, np.zeros(3)
    for a, expect in [(-1e-4, 0.0), (2e-4, 0.0), (1e-3, min(g * 6e-3, 1.0)),
                      (3e-3, 0.36), (2e-2, 1.0)]:
        gu = -a * np.eye(3)                       # div u = -3a
        Q, J, _ = build_first_moments(rho, u, p, np.zeros(3), gu, np.zeros(3), 0.0, 0.0,
                                      np.full(5, P.omega[0]), 1.4)
        _, info = oracle.cell(P, pops_with_moments(Q, J))
        s = 6 * a                                 # -div u / cs with cs = 1/2
        want = 0.0 if (a <= 0 or s <= jmin) else min(g * s, 1.0)
        assert info.chi == pytest.approx(want, abs=1e-12)
        assert info.chi == pytest.approx(expect, abs=1e-12)


def test_gated_collision_is_bgk_off_the_sensor_and_regularized_on_it():
    """Sensor-gated collision (the reading of Sec. 2.2 in which the sensor activates the
    regularized operator in place of BGK), checked by the post-collision moments of an
    inviscid cell whose populations carry a second-moment non-equilibrium part:
      chi = 0 (expansion): BGK keeps (1 - omega) of it, Sigma f* c_x^2 - cs^2 Q =
                           (1 - omega)(Sigma f c_x^2 - cs^2 Q);
      chi > 0 (compression): the regularized collision discards it (Sec. 2.5);
    and in both the first moment is J + omega_r (Phi - J) with Phi the Euler flux and
    omega_r = omega (BGK) or omega_h = omega - chi (omega - omega_min) (Listing 2)."""
    g, jmin, om_min = 20.0, 3e-3, 1.0
    P = lattice_P(mu_ref=0.0, sensor_gain=g, J_min=jmin, omega_min=om_min, collision=2)
    om = P.omega[0]
    rho, p, u = 1.0, 0.5, np.array([0.03, -0.02, 0.01])
    for a in (-1e-3, 3e-3):                          # expansion, compression (chi = 0.36)
        gu = -a * np.eye(3)
        Q, J, _ = build_first_moments(rho, u, p, np.zeros(3), gu, np.zeros(3), 0.0, 0.0,
                                      np.full(5, om), 1.4)
        f = pops_with_moments(Q, J)
        dev = 1e-3 * np.arange(1, 6)                 # second-moment deviation per field
        for k in range(5):
            f[7 * k + 1] += dev[k]
            f[7 * k + 2] += dev[k]
            f[7 * k + 0] -= 2 * dev[k]              # Q and J unchanged
        fstar, info = oracle.cell(P, f)
        chi = 0.0 if 6 * a <= jmin else min(g * 6 * a, 1.0)
        assert info.chi == pytest.approx(chi, abs=1e-12)
        _, Phi = euler_flux(rho, u, p, 1.4)
        om_r = om - chi * max(om - om_min, 0.0)
        for k in range(5):
            Pin = f[7 * k + 1] + f[7 * k + 2] - CS2 * Q[k]
            Pout = fstar[7 * k + 1] + fstar[7 * k + 2] - CS2 * Q[k]
            want = 0.0 if chi > 0 else (1.0 - om) * Pin
            assert Pout == pytest.approx(want, abs=1e-14)
            Jout = CI.T @ fstar[7 * k:7 * k + 7]
            np.testing.assert_allclose(Jout, J[k] + om_r * (Phi[k] - J[k]), atol=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_regularized_outgoing_set_lies_in_the_span_of_four_moments(seed):
    """Sec. 2.5: the regularized collision keeps only the equilibrium and the first-moment
    non-equilibrium part, so each field's outgoing populations are w_i (Q*_k + c_i . J*_k / cs^2)
    with Q*_k, J*_k their own zeroth and first moments -- four numbers per field, whatever
    second-moment non-equilibrium the incoming set carries (the fact that lets the state be
    stored as 20 moments per cell).  BGK keeps (1 - omega) of that part, so its outgoing set
    leaves the span: the check can fail."""
    rng = np.random.default_rng(40 + seed)
    rho, p = rng.uniform(0.7, 1.5), rng.uniform(0.1, 0.5)
    u = rng.uniform(-0.1, 0.1, 3)
    gu = rng.uniform(-2e-3, 2e-3, (3, 3))
    gr, gT = rng.uniform(-1e-3, 1e-3, 3), rng.uniform(-1e-3, 1e-3, 3)
    out = {}
    for coll in (inputs.COLL_RLB_SENSOR, inputs.COLL_BGK):
        P = lattice_P(mu_ref=0.05, collision=coll)
        Q, J, _ = build_first_moments(rho, u, p, gr, gu, gT, 0.05, 0.07, np.full(5, P.omega[0]), 1.4)
        f = pops_with_moments(Q, J)
        f += 1e-3 * rng.standard_normal(35) * np.repeat([1, 1, 1, 1, 2], 7)  # every moment perturbed
        fstar, _ = oracle.cell(P, f)
        worst = 0.0
        for k in range(5):
            fk = fstar[7 * k:7 * k + 7]
            Qs, Js = fk.sum(), CI.T @ fk
            span = WI * (Qs + CI @ Js / CS2)
            worst = max(worst, np.abs(fk - span).max())
        out[coll] = worst
    assert out[inputs.COLL_RLB_SENSOR] <= 1e-15
    assert out[inputs.COLL_BGK] > 1e-6


def test_gated_collision_without_sensor_gain_is_bgk():
    """With gain 0 the sensor never fires, so the gated collision is BGK on every cell."""
    c = inputs.random_smooth(10, 7, 5, seed=4)
    runs = []
    for coll, gain in ((2, 0.0), (0, 0.0)):
        o = oracle.Oracle(c.params.replace(collision=coll, sensor_gain=gain))
        o.init_primitive(c.rho, c.u, c.p)
        o.step(15)
        runs.append(o.f.copy())
    assert np.array_equal(runs[0], runs[1])


# ---- invariants ----------------------------------------------------------------------------
@pytest.mark.parametrize("collision", [0, 1, 2])
def test_conservation_on_periodic_domain(collision):
    c = inputs.random_smooth(8, 6, 5, seed=1, collision=collision)
    o = oracle.Oracle(c.params)
    o.init_primitive(c.rho, c.u, c.p)
    Q0 = o.conserved_lattice()
    o.step(40)
    Q1 = o.conserved_lattice()
    scale = np.abs(Q0).max(1)
    drift = np.abs(Q1.sum(1) - Q0.sum(1)) / (scale * Q0.shape[1])
    assert drift.max() < 1e-14
    assert np.abs(Q1 - Q0).max() > 1e-4             # the flow did evolve


@pytest.mark.parametrize("collision", [0, 1, 2])
def test_uniform_state_is_invariant(collision):
    c = inputs.uniform(6, 5, 4, collision=collision)
    o = oracle.Oracle(c.params)
    o.init_primitive(c.rho, c.u, c.p)
    f0 = o.f.copy()
    o.step(20)
    assert np.abs(o.f - f0).max() < 1e-14


# ---- exact solutions -----------------------------------------------------------------------
def test_sod_exact_solver_matches_textbook_star_state():
    gold = json.load(open(os.path.join(GOLDEN, "sod_toro.json")))
    ps, us = exact.sod_star((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    tol = gold["tolerance_abs"]
    assert ps == pytest.approx(gold["p_star"], abs=tol)
    assert us == pytest.approx(gold["u_star"], abs=tol)
    x = np.array([0.5 + 0.2 * (us - 1e-3), 0.5 + 0.2 * (us + 1e-3)])
    r, u, p = exact.sod_exact(x, 0.2)
    assert r[0] == pytest.approx(gold["rho_star_left"], abs=tol)
    assert r[1] == pytest.approx(gold["rho_star_right"], abs=tol)


def test_sod_exact_solver_satisfies_jump_conditions():
    g = 1.4
    ps, us = exact.sod_star((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    # right shock: Rankine-Hugoniot mass, momentum and energy fluxes in the shock frame
    x = np.linspace(0.0, 1.0, 20001)
    r, u, p = exact.sod_exact(x, 0.2)
    i = np.argmax(np.abs(np.diff(p)) * (x[1:] > 0.8))
    S = (x[i] - 0.5) / 0.2
    (r1, u1, p1), (r2, u2, p2) = (r[i + 1], u[i + 1], p[i + 1]), (r[i], u[i], p[i])
    w1, w2 = u1 - S, u2 - S
    assert r1 * w1 == pytest.approx(r2 * w2, rel=2e-3)
    assert r1 * w1 * w1 + p1 == pytest.approx(r2 * w2 * w2 + p2, rel=2e-3)
    h = lambda rr, pp, ww: g / (g - 1) * pp / rr + 0.5 * ww * ww
    assert h(r1, p1, w1) == pytest.approx(h(r2, p2, w2), rel=2e-3)
    # rarefaction: isentropic and left Riemann invariant u + 2c/(gamma-1) constant
    fan = (x > 0.5 - 0.2 * 1.18) & (x < 0.5 - 0.2 * 0.0)
    fan &= (u > 1e-3) & (u < us - 1e-3)
    c = np.sqrt(g * p[fan] / r[fan])
    np.testing.assert_allclose(p[fan] / r[fan] ** g, 1.0, rtol=1e-10)
    np.testing.assert_allclose(u[fan] + 2 * c / (g - 1), 2 * math.sqrt(g) / (g - 1), rtol=1e-10)


def test_becker_profile_solves_the_viscous_shock_ode():
    g, M, mu = 1.4, 2.0, 2e-3
    x = np.linspace(0.45, 0.55, 4001)
    r, u, p = exact.becker_profile(x, M, mu, 0.5)
    (r1, u1, p1), (r2, u2, p2) = inputs.becker_states(M, g)
    # end states are the Rankine-Hugoniot states
    far = exact.becker_profile(np.array([-1.0, 2.0]), M, mu, 0.5)
    np.testing.assert_allclose([far[0][0], far[1][0], far[2][0]], [r1, u1, p1], rtol=1e-9)
    np.testing.assert_allclose([far[0][1], far[1][1], far[2][1]], [r2, u2, p2], rtol=1e-9)
    # steady 1-D NSF: mass flux, momentum flux rho u^2 + p - (4/3) mu u' constant
    du = np.gradient(u, x)
    np.testing.assert_allclose(r * u, r1 * u1, rtol=1e-9)
    mom = r * u * u + p - 4.0 / 3.0 * mu * du
    np.testing.assert_allclose(mom[5:-5], r1 * u1 * u1 + p1, rtol=2e-5)
    # energy flux (E + p) u - (4/3) mu u u' - kappa T' with Pr = 3/4
    kappa = mu * (g / (g - 1)) / 0.75
    T = p / r
    E = p / (g - 1) + 0.5 * r * u * u
    en = (E + p) * u - 4.0 / 3.0 * mu * u * du - kappa * np.gradient(T, x)
    E1 = p1 / (g - 1) + 0.5 * r1 * u1 * u1
    np.testing.assert_allclose(en[5:-5], (E1 + p1) * u1, rtol=2e-5)


def sod_errors(nx, collision=inputs.COLL_RLB_SENSOR):
    c = inputs.sod(nx, steps=int(round(0.2 / (0.08 / nx))))
    o = oracle.Oracle(c.params.replace(collision=collision))
    o.init_primitive(c.rho, c.u, c.p)
    o.step(c.meta["steps"])
    rho, u, p, _ = o.primitive()
    x = c.meta["x"]
    re, ue, pe = exact.sod_exact(x, 0.2)
    m = (x > 0.05) & (x < 0.95)
    L2 = lambda a, b: math.sqrt(((a - b)[m] ** 2).sum() / (b[m] ** 2).sum())
    return L2(rho, re), L2(p, pe), L2(u[0], ue)


@pytest.mark.parametrize("collision", [inputs.COLL_RLB_SENSOR, inputs.COLL_RLB_GATED])
def test_sod_tube_against_exact_riemann_solution(collision):
    """Sod tube, 400 cells, 1000 steps to t = 0.2 (dt/dx = 0.08): inviscid limit; the
    regularized collision of Alg. 1 and the gated reading of Sec. 2.2 alike."""
    er, ep, eu = sod_errors(400, collision)
    assert er < 5e-2 and ep < 5e-2 and eu < 1e-1


@pytest.mark.slow
def test_sod_tube_error_comparable_to_paper_table():
    gold = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))["sod_conv"]
    er, ep, eu = sod_errors(750)
    e400 = sod_errors(400)
    assert er < e400[0] and ep < e400[1]
    # same order as the paper's N = 750 row (within a factor 2.5)
    assert er < 2.5 * gold["rho"][0] and ep < 2.5 * gold["p"][0] and eu < 2.5 * gold["u"][0]


def becker_error(nx, cpf, collision=inputs.COLL_RLB_SENSOR):
    # omega tied to dt: tau - 1/2 proportional to dt, omega = 1.99 at 128 cells per front
    om = 1.0 / (0.5 + (1.0 / 1.99 - 0.5) * 128.0 / cpf)
    c = inputs.becker(nx, cells_per_front=cpf, omega=om, cfl_max=0.1)
    x = c.meta["x"]
    re, ue, pe = exact.becker_profile(x, 2.0, c.meta["mu"], 0.5)
    o = oracle.Oracle(c.params.replace(collision=collision))
    o.init_primitive(re, np.stack([ue, 0 * ue, 0 * ue]), pe)
    o.step(int(1.0 / c.params.dt))
    rho, u, p, _ = o.primitive()
    from scipy.optimize import minimize_scalar
    err = lambda x0: np.sqrt(((rho - exact.becker_profile(x, 2.0, c.meta["mu"], x0)[0]) ** 2).sum()
                             / (re ** 2).sum())
    x0 = minimize_scalar(err, bounds=(0.45, 0.55), method="bounded",
                         options={"xatol": 1e-12}).x
    r2, u2, p2 = exact.becker_profile(x, 2.0, c.meta["mu"], x0)
    L2 = lambda a, b: math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())
    return L2(rho, r2), L2(p, p2), L2(u[0], u2)


@pytest.mark.parametrize("collision", [inputs.COLL_RLB_SENSOR, inputs.COLL_RLB_GATED])
def test_becker_viscous_shock_converges_at_second_order(collision):
    """Becker closed form, 8 -> 16 cells across the front: the error falls at about second
    order and stays below the paper's Tab. becker_conv rows (both readings of the collision)."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))["becker_conv"]
    e8 = becker_error(128, 8, collision)
    e16 = becker_error(256, 16, collision)
    for a, b in zip(e8, e16):
        assert math.log2(a / b) > 1.5
    assert e8[0] < gold["rho"][0] and e16[0] < gold["rho"][1]
    assert e8[2] < gold["u"][0] and e16[2] < gold["u"][1]


@pytest.mark.parametrize("n,tol", [(32, 0.02), (64, 0.006)])
def test_low_mach_taylor_green_decay_rate(n, tol):
    """2-D Taylor-Green at Ma = 0.05, BGK at omega = 2 (no numerical viscosity): kinetic
    energy decays as exp(-4 nu k^2 t) over one e-fold, all of it from the reconstructed
    stress."""
    c = inputs.tgv2d(n, mach=0.05, nu_lat=0.01 if n == 32 else 0.02)
    o = oracle.Oracle(c.params)
    o.init_primitive(c.rho, c.u, c.p)
    rate = 4 * c.meta["nu"] * c.meta["k"] ** 2
    ke = lambda Q: (0.5 * (Q[1] ** 2 + Q[2] ** 2) / Q[0]).sum()
    k0 = ke(o.conserved())
    nsteps = int(1.0 / rate / c.params.dt)
    o.step(nsteps)
    measured = -math.log(ke(o.conserved()) / k0) / (nsteps * c.params.dt)
    assert measured / rate == pytest.approx(1.0, abs=tol)
