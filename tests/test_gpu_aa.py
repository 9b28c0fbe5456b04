"""One-buffer in-place streaming (AA pattern): half the population memory, the same collisions.

With the initial state written in swapped slots, odd steps (pull from the neighbours' opposite
slots, push to the neighbours) and even steps (own slots, swapped on write) apply the
collisions of the two-buffer pull sweep to the same inputs.  The kernels are separate
instantiations of the one collide, whose rounding is fixed by its source (no compiler
contraction in the sweep file), so the results are bit for bit the two-buffer run's (every
storage type, 30 steps), and a one-buffer run is bitwise reproducible against itself and
across a checkpoint.  Every case also matches the FP64 oracle
(rel L-inf 1e-5 smooth / rel L1 1e-4 tubes for FP32 storage)."""
import numpy as np
import pytest

from paper_2609_16361_b300 import capi, inputs
from tests.common import run_oracle
from tests.test_gpu_batch import oracle_gate

pytestmark = pytest.mark.gpu


def run(case, steps, streaming, diag=False):
    prm = case.params.replace(streaming=streaming)
    d = capi.Domain(prm)
    d.init(case.rho, case.u, case.p)
    if diag:
        d.step(steps - 1)
        d.step_diag()
    else:
        d.step(steps)
    return d


def cases():
    om = inputs.becker_tied_omega(8.0)
    return [inputs.tgv3d(24), inputs.tgv3d(20, storage=inputs.STORE_F16),
            inputs.random_smooth(40, 21, 7, seed=5, collision=inputs.COLL_BGK),
            inputs.sod(400), inputs.sod(100, steps=250, storage=inputs.STORE_BF16),
            inputs.becker(128, cells_per_front=8, omega=om, cfl_max=0.1, ny=4, nz=4),
            inputs.random_smooth(1, 1, 1, seed=2)]


@pytest.mark.parametrize("steps", [1, 2, 7, 30])
def test_in_place_equals_two_buffers(steps):
    for c in cases():
        a = run(c, steps, 0)
        b = run(c, steps, 1)
        assert b.steps == steps
        assert np.array_equal(b.conserved(), a.conserved()), (c.params.name, steps)
        cells = np.arange(c.params.ncells)
        assert np.array_equal(capi.grlb_read_cells(b.h, cells), capi.grlb_read_cells(a.h, cells))
        b2 = run(c, steps, 1)
        assert np.array_equal(b.conserved(), b2.conserved())
        for d in (a, b, b2):
            d.close()


@pytest.mark.parametrize("steps", [7, 100])
def test_in_place_matches_the_oracle(steps):
    for c in cases():
        b = run(c, steps, 1)
        R = run_oracle(c, steps).conserved()
        Q = b.conserved()
        if c.params.ncells == 1:   # a single cell: no flow, compare with a floor on the scale
            scale = np.maximum(np.abs(R).max(1), 1e-3)
            assert np.all(np.abs(Q - R).max(1) / scale <= 1e-5)
        else:
            ok, err = oracle_gate(c, Q, R)
            assert ok, (c.params.name, steps, err)
        b.close()


def test_in_place_diagnostics_and_memory():
    c = inputs.tgv3d(32)
    a = run(c, 11, 0, diag=True)
    b = run(c, 11, 1, diag=True)
    ga, gb = a.diag(), b.diag()
    np.testing.assert_allclose(gb["totals"][[0, 4]], ga["totals"][[0, 4]], rtol=1e-6)
    # momentum totals cancel to ~1e-6 of sums of |m| ~ 1e3: compare absolutely
    np.testing.assert_allclose(gb["totals"][1:4], ga["totals"][1:4], atol=1e-5)
    for k in ("ke", "eps_s", "eps_d", "rho_min", "p_min"):
        np.testing.assert_allclose(gb[k], ga[k], rtol=1e-5, err_msg=k)
    pops = 35 * 32 ** 3 * 4
    assert capi.lib().grlb_device_bytes(a.h) - capi.lib().grlb_device_bytes(b.h) == pops
    assert capi.grlb_bytes_for(c.params.replace(streaming=1)) == capi.lib().grlb_device_bytes(b.h)


def test_in_place_checkpoint_resume_at_odd_step():
    c = inputs.tgv3d(16)
    a = run(c, 13, 1)
    ck = capi.grlb_save(a.h)
    a.step(8)
    b = capi.Domain(c.params.replace(streaming=1))
    capi.grlb_load(b.h, ck)
    b.step(8)
    assert np.array_equal(a.conserved(), b.conserved())
    ref = run(c, 21, 0)
    assert np.array_equal(b.conserved(), ref.conserved())


def test_in_place_refuses_sources_and_batches():
    c = inputs.tgv3d(8)
    d = capi.Domain(c.params.replace(streaming=1))
    with pytest.raises(capi.GrlbError):
        capi.grlb_set_source_device(d.h, 1)
    with pytest.raises(capi.GrlbError):
        capi.grlb_batch_create([d.h], schedule=capi.SCHED_TABLE_CONST)
    b = capi.grlb_batch_create([d.h])          # the concurrent schedule takes it
    capi.grlb_batch_step(b, 3)
    capi.grlb_batch_destroy(b)
    assert d.steps == 3
