"""Moment storage (grlb_params.streaming = 2): the state of a regularized-collision domain kept
as the 20 moments (Q_k, J*_k) of each cell's outgoing set instead of its 35 populations.

The regularized collision of Algorithm 1 leaves every field's outgoing set on w_i (Q_k + c_i .
J*_k / cs^2), each population formed from Q_k and one component of J*_k by the same FP32
operations, so storing the moments and rebuilding the populations at the pull is an exact
re-encoding: the moment-storage run must equal the population run bit for bit -- populations
(through the point probes), conserved fields, diagnostics, spectra, checkpoints -- for periodic
boxes, ragged linear launches, Dirichlet tubes, the Chapman-Enskog start, batches and the
staged upload; and it must refuse what it cannot represent (BGK and gated cells keep parts of
the populations outside the moments; 16-bit storage; sources; the allocation-free sweep).  The
z-slab exchange of moment slabs is tested in test_gpu_slabs.py."""
import numpy as np
import pytest

import oracle
from paper_2609_16361_b300 import capi, inputs
from tests.common import rel_l1, rel_linf

pytestmark = pytest.mark.gpu


def run(case, steps, streaming, ce=None, diag=False):
    d = capi.Domain(case.params.replace(streaming=streaming))
    d.init(case.rho, case.u, case.p, ce_init=ce)
    if diag:
        d.step(steps - 1)
        d.step_diag()
    else:
        d.step(steps)
    return d


CASES = {
    "tgv32 (tiled, 32 x 4)": lambda: inputs.tgv3d(32),
    "128x8x6 (whole-brick rows: L2 prefetch)": lambda: inputs.random_smooth(128, 8, 6, seed=8),
    "ragged 40x21x7 (linear)": lambda: inputs.random_smooth(40, 21, 7, seed=3),
    "sod 400 (Dirichlet ghosts)": lambda: inputs.sod(400),
    "becker 128x4x4": lambda: inputs.becker(128, ny=4, nz=4),
    "tgv24 Mach 0.5 Re 100": lambda: inputs.tgv3d(24, mach=0.5, re=100.0),
    "single cell": lambda: inputs.random_smooth(1, 1, 1, seed=2),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("steps", [1, 8, 9, 50])
def test_moment_storage_is_bitwise_the_population_run(name, steps):
    """1 step, one graph of 8, a graph plus one, and 50 steps with the diagnostic sweep last."""
    c = CASES[name]()
    a = run(c, steps, 0, diag=steps == 50)
    b = run(c, steps, 2, diag=steps == 50)
    assert b.steps == a.steps == steps
    cells = np.arange(c.params.ncells)
    assert np.array_equal(capi.grlb_read_cells(b.h, cells), capi.grlb_read_cells(a.h, cells))
    assert np.array_equal(b.conserved(), a.conserved())
    # a checkpoint keeps its layout: it loads only into a domain of the same kind
    with pytest.raises(capi.GrlbError):
        capi.grlb_load(a.h, capi.grlb_save(b.h))
    with pytest.raises(capi.GrlbError):
        capi.grlb_load(b.h, capi.grlb_save(a.h))
    ra, rb = a.primitive(), b.primitive()
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)
    if steps == 50:
        assert_same_diagnostics(a.diag(), b.diag())
    a.close()
    b.close()


def assert_same_diagnostics(ga, gb):
    """Counters and minima exactly; the sums to FP32 rounding: moment storage launches 32 x 4
    tiles where the population sweep takes 128 x 1, so the warp-level FP32 partial sums group
    other cells (bitwise equal where the tiles agree)."""
    for k in ("rho_min", "p_min", "n_floor", "n_nan", "n_sensor", "step"):
        assert ga[k] == gb[k], k
    for k in ("totals", "ke", "eps_s", "eps_d"):
        np.testing.assert_allclose(np.asarray(gb[k]), np.asarray(ga[k]), rtol=1e-6, atol=0, err_msg=k)


def test_moment_storage_matches_the_oracle():
    """The parity bars of the sweep, directly against the FP64 oracle (smooth and shocked)."""
    for c, steps, bound, norm in ((inputs.tgv3d(32), 100, 1e-5, rel_linf),
                                  (inputs.sod(400), 100, 1e-4, rel_l1)):
        d = run(c, steps, 2)
        o = oracle.Oracle(c.params)
        o.init_primitive(c.rho, c.u, c.p)
        o.step(steps)
        err = norm(d.conserved(), o.conserved())
        assert np.all(err <= bound), (c.params.name, err)
        d.close()


def test_chapman_enskog_start_and_spectra():
    c = inputs.tgv3d(32, mach=0.5, re=100.0)
    a, b = run(c, 7, 0, ce=True), run(c, 7, 2, ce=True)
    assert np.array_equal(b.conserved(), a.conserved())
    Ea, sa = a.spectral()
    Eb, sb = b.spectral()
    assert np.array_equal(Ea, Eb) and np.array_equal(sa, sb)
    a.close()
    b.close()


def test_checkpoint_staging_and_finiteness_scan():
    torch = pytest.importorskip("torch")
    c = inputs.tgv3d(16)
    other = inputs.tgv3d(16, mach=0.8)
    b = run(c, 5, 2)
    ck = capi.grlb_save(b.h)
    assert ck.size == 32 + 20 * 4 * 16 ** 3  # 20 FP32 moments per cell (whole bricks: 4096 cells)
    b.step(10)
    r = capi.Domain(c.params.replace(streaming=2))
    capi.grlb_load(r.h, ck)
    r.step(10)
    assert np.array_equal(r.conserved(), b.conserved())
    # staged upload into a moment domain equals the direct initialisation
    capi.grlb_stage_primitive(r.h, other.rho, other.u, other.p)
    capi.grlb_init_from_stage(r.h)
    r.step(3)
    direct = capi.Domain(c.params.replace(streaming=2))
    direct.init(other.rho, other.u, other.p)
    direct.step(3)
    assert np.array_equal(r.conserved(), direct.conserved())
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.grlb_check_finite(r.h, flag.data_ptr())
    torch.cuda.synchronize()
    assert int(flag.item()) == 0
    for d in (b, r, direct):
        d.close()


def test_moment_domains_in_a_batch_run_their_own_sweep():
    cases = [inputs.tgv3d(16), inputs.becker(128, ny=4, nz=4), inputs.tgv3d(20, storage=inputs.STORE_F16)]
    prms = [cases[0].params.replace(streaming=2), cases[1].params.replace(streaming=2), cases[2].params]
    doms = [capi.Domain(p) for p in prms]
    for d, c in zip(doms, cases):
        d.init(c.rho, c.u, c.p)
    for sched in (capi.SCHED_CONCURRENT, capi.SCHED_TABLE_CONST):
        b = capi.grlb_batch_create([d.h for d in doms], schedule=sched)
        capi.grlb_batch_step(b, 6)
        capi.grlb_batch_destroy(b)
    for d, c, p in zip(doms, cases, prms):
        solo = capi.Domain(p)
        solo.init(c.rho, c.u, c.p)
        solo.step(12)
        assert np.array_equal(d.conserved(), solo.conserved()), p.name
        solo.close()
        d.close()


def test_what_moments_cannot_hold_is_refused():
    torch = pytest.importorskip("torch")
    base = inputs.tgv3d(16).params.replace(streaming=2)
    for bad in (base.replace(collision=inputs.COLL_BGK), base.replace(collision=inputs.COLL_RLB_GATED),
                base.replace(storage=inputs.STORE_F16), base.replace(storage=inputs.STORE_BF16)):
        with pytest.raises(capi.GrlbError):
            capi.Domain(bad)
    d = capi.Domain(base)
    S = torch.zeros((5, base.ncells), dtype=torch.float32, device="cuda")
    with pytest.raises(capi.GrlbError):
        capi.grlb_set_source_device(d.h, S.data_ptr())
    with pytest.raises(capi.GrlbError):
        capi.grlb_step_diag_noalloc(base, S.data_ptr(), S.data_ptr(), S.data_ptr(), None)
    d.close()


def test_full_size_moment_storage_is_bitwise_the_population_run():
    """The headline configuration (256^3 Taylor-Green, FP32, regularized collision) after 60
    sweeps in the launch configuration the benchmark times: every probed population of 3000
    sampled cells and every conserved value equal."""
    torch = pytest.importorskip("torch")
    prm, rho, u, p = inputs.tgv3d_device(256)
    out = []
    rng = np.random.default_rng(3)
    cells = np.unique(np.concatenate([rng.integers(0, prm.ncells, 3000), [0, prm.ncells - 1]]))
    for streaming in (0, 2):
        d = capi.Domain(prm.replace(streaming=streaming))
        capi.grlb_init_primitive_device(d.h, rho.data_ptr(), u.data_ptr(), p.data_ptr())
        d.step(59)
        d.step_diag()
        out.append((capi.grlb_read_cells(d.h, cells), d.conserved(), d.diag()))
        d.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert_same_diagnostics(out[0][2], out[1][2])
