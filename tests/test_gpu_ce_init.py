"""GPU Chapman-Enskog initialisation (grlb_set_init_mode(d, 1)) against the FP64 oracle.

Tolerances: the non-equilibrium part the initialisation adds (population difference between
the Chapman-Enskog and the equilibrium start) agrees to 1e-4 of its largest magnitude per
field -- FP32 populations carry ~6e-8 of |f|, and the part is ~1e-2 of |f| on these flows --;
after 100 sweeps the conserved fields meet the sweep parity bar (rel L-inf 1e-5 smooth,
rel L1 1e-4 across shocks).
"""
import numpy as np
import pytest

import oracle
from oracle import spectral
from paper_2609_16361_b300 import capi, inputs
from tests.common import decode_populations, rel_l1, rel_linf

pytestmark = pytest.mark.gpu


def gpu_start(case, ce, steps=0, streaming=0):
    prm = case.params.replace(streaming=streaming)
    d = capi.Domain(prm)
    d.init(case.rho, case.u, case.p, ce_init=ce)
    if steps:
        d.step(steps)
    return d


def oracle_start(case, ce, steps=0):
    o = oracle.Oracle(case.params)
    o.init_primitive(case.rho, case.u, case.p, ce_init=ce)
    if steps:
        o.step(steps)
    return o


def neq_part_gpu(case):
    a, b = gpu_start(case, True), gpu_start(case, False)
    fa = decode_populations(capi.grlb_save(a.h), case.params)
    fb = decode_populations(capi.grlb_save(b.h), case.params)
    a.close()
    b.close()
    return fa - fb


def assert_neq_close(case):
    dg = neq_part_gpu(case)
    do = oracle_start(case, True).f - oracle_start(case, False).f
    for k in range(5):
        sl = slice(7 * k, 7 * k + 7)
        scale = np.abs(do[sl]).max()
        if scale == 0.0:
            assert np.abs(dg[sl]).max() == 0.0
            continue
        assert np.abs(dg[sl] - do[sl]).max() <= 1e-4 * scale, (k, np.abs(dg[sl] - do[sl]).max(), scale)


def test_taylor_green_neq_part_matches_oracle():
    assert_neq_close(inputs.tgv3d(32, mach=1.25, re=100.0))


def test_random_smooth_ragged_neq_part_matches_oracle():
    assert_neq_close(inputs.random_smooth(40, 21, 7, seed=9))


@pytest.mark.parametrize("which", ["sod", "becker"])
def test_tube_with_ghost_states_neq_part_matches_oracle(which):
    assert_neq_close(inputs.sod(128) if which == "sod" else inputs.becker(256, 3.0))


def test_uniform_field_is_bitwise_the_plain_start():
    c = inputs.uniform(33, 5, 3)
    a, b = gpu_start(c, True), gpu_start(c, False)
    assert np.array_equal(capi.grlb_save(a.h), capi.grlb_save(b.h))
    a.close()
    b.close()


@pytest.mark.parametrize("fmu,steps", [(0.001, 40), (0.9, 100)])
def test_parity_after_steps(fmu, steps):
    """At f_mu = 0.001 (omega = 1.9998) the regularized collision with the linear equilibrium
    amplifies perturbations (the instability near omega = 2): in the FP64 oracle itself a
    relative perturbation of 6e-8 (FP32 rounding) of the initial populations grows to 1.4e-6
    after 50 steps and 9e-5 after 100, with either start; at f_mu = 0.9 it stays below 6e-6.
    The omega = 2 case is therefore compared after 40 steps, the damped one after 100."""
    c = inputs.tgv3d(32, mach=0.5, re=100.0, fmu=fmu)
    d = gpu_start(c, True, steps)
    o = oracle_start(c, True, steps)
    err = rel_linf(d.conserved(), o.conserved())
    assert np.all(err <= 1e-5), err
    d.close()


def test_sod_parity_after_100_steps():
    c = inputs.sod(400)
    d = gpu_start(c, True, 100)
    o = oracle_start(c, True, 100)
    err = rel_l1(d.conserved(), o.conserved())
    assert np.all(err <= 1e-4), err
    d.close()


def test_one_buffer_layout():
    c = inputs.random_smooth(32, 32, 32, seed=3)
    a = gpu_start(c, True, 7, streaming=0)
    b = gpu_start(c, True, 7, streaming=1)
    err = rel_linf(b.conserved(), a.conserved())
    assert np.all(err <= 1e-6), err
    a.close()
    b.close()


def test_cell_local_dissipation_does_not_alternate():
    """omega = 1.9998 (f_mu = 0.001, the 256^3 setting): with the Chapman-Enskog start
    the cell-local eps_s of the diagnostic sweep tracks the spectral one at even and odd steps;
    the equilibrium start reads ~0 at even steps."""
    c = inputs.tgv3d(64, mach=0.5, re=100.0, fmu=0.001)
    out = {}
    for ce in (True, False):
        d = gpu_start(c, ce)
        ratios = []
        for n in (49, 0):
            d.step(n)
            d.step_diag()
            cell = d.diag()["eps_s"]
            _, sp = d.spectral()
            ratios.append(cell / sp["eps_s"])
        out[ce] = ratios
        d.close()
    assert all(abs(r - 1.0) < 0.05 for r in out[True]), out
    assert out[False][0] < 0.1 and out[False][1] > 2.0, out


def test_f16_storage_close_to_oracle():
    c = inputs.tgv3d(32, mach=0.5, re=100.0, storage=inputs.STORE_F16)
    d = gpu_start(c, True, 20)
    o = oracle_start(c, True, 20)
    err = rel_linf(d.conserved(), o.conserved())
    assert np.all(err <= 1e-2), err
    d.close()


def test_rejects_bad_mode():
    c = inputs.uniform(8, 4, 4)
    d = capi.Domain(c.params)
    with pytest.raises(capi.GrlbError):
        capi.grlb_set_init_mode(d.h, 2)
    d.close()
