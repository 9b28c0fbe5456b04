"""Batches: many uneven domains (Becker tubes, Taylor-Green boxes, mixed storage and
collision) advanced by one call, under the three schedules: concurrent single-domain sweeps
(default; bitwise grlb_step), and one launch per step over all small domains with the records
in the constant table or in device memory (tile table).

* A domain's batched result is bitwise independent of the other domains in the batch (alone
  in a batch == in the mix), under every schedule.
* It is bitwise the solo run under every schedule: the table kernels read the domain constants
  from other memory spaces than the single-domain sweep, but the collide's rounding is fixed by
  its source (no compiler contraction in the sweep file).
* Every domain of the mix matches the FP64 oracle after 100 batched steps: relative L-inf
  <= 1e-5 for smooth fields and relative L1 <= 1e-4 for the shock tubes (FP32 storage; the
  FP16 / BF16 domains within the loose bounds of their other oracle comparisons).
* Inactive domains do not move."""
import numpy as np
import pytest

from paper_2609_16361_b300 import capi, inputs
from tests.common import rel_l1, rel_linf, run_oracle

pytestmark = pytest.mark.gpu


def mixed_cases():
    om = 1.0 / (0.5 + (1.0 / 1.99 - 0.5) * 128.0 / 8)
    return [
        inputs.tgv3d(16),
        # Mach 0.5 needs dt = 0.05 dx to keep |u| + c below 1/4 per step (sensor-gated collision)
        inputs.tgv3d(24, mach=0.5, cfl=0.05, collision=inputs.COLL_RLB_GATED),
        inputs.becker(128, cells_per_front=8, omega=om, cfl_max=0.1, ny=4, nz=4),
        inputs.becker(200, mach=3.0, cells_per_front=8, omega=om, cfl_max=0.1),
        inputs.random_smooth(40, 21, 7, seed=5, collision=inputs.COLL_BGK),
        inputs.tgv3d(20, storage=inputs.STORE_F16),
        inputs.sod(100, steps=250, storage=inputs.STORE_BF16),
    ]


def solo(case, n):
    d = capi.Domain(case.params)
    d.init(case.rho, case.u, case.p)
    d.step(n)
    Q = d.conserved()
    raw = capi.grlb_save(d.h)[32:]
    d.close()
    return Q, raw


SCHEDULES = [capi.SCHED_CONCURRENT, capi.SCHED_TABLE_CONST, capi.SCHED_TABLE]
TABLES = [capi.SCHED_TABLE_CONST, capi.SCHED_TABLE]


def batched_alone(case, n, block_x=0, use_graph=1, schedule=capi.SCHED_TABLE_CONST):
    d = capi.Domain(case.params)
    d.init(case.rho, case.u, case.p)
    b = capi.grlb_batch_create([d.h], block_x=block_x, use_graph=use_graph, schedule=schedule)
    capi.grlb_batch_step(b, n)
    raw = capi.grlb_save(d.h)[32:]
    capi.grlb_batch_destroy(b)
    d.close()
    return raw


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("use_graph,nsteps,block_x", [(1, 30, 0), (0, 17, 64), (1, 13, 32)])
def test_batch_equals_solo_runs(use_graph, nsteps, block_x, schedule):
    cases = mixed_cases()
    doms = []
    for c in cases:
        d = capi.Domain(c.params)
        d.init(c.rho, c.u, c.p)
        doms.append(d)
    b = capi.grlb_batch_create([d.h for d in doms], block_x=block_x, use_graph=use_graph,
                               schedule=schedule)
    # two calls, so the second starts from each domain's flipped buffer
    k = nsteps // 2
    capi.grlb_batch_step(b, k)
    capi.grlb_batch_step(b, nsteps - k)
    for c, d in zip(cases, doms):
        assert d.steps == nsteps
        raw = capi.grlb_save(d.h)[32:]
        # alone in a batch == in the mix, bitwise
        assert np.array_equal(raw, batched_alone(c, nsteps, block_x, use_graph, schedule)), c.params.name
        Q_ref, raw_ref = solo(c, nsteps)
        assert np.array_equal(raw, raw_ref), (c.params.name, schedule)
        assert np.array_equal(d.conserved(), Q_ref), (c.params.name, schedule)
    capi.grlb_batch_destroy(b)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_inactive_domains_do_not_move(schedule):
    cases = mixed_cases()[:3]
    doms = []
    for c in cases:
        d = capi.Domain(c.params)
        d.init(c.rho, c.u, c.p)
        doms.append(d)
    b = capi.grlb_batch_create([d.h for d in doms], use_graph=1, schedule=schedule)
    before = capi.grlb_save(doms[1].h)[32:].copy()
    capi.grlb_batch_set_active(b, [1, 0, 1])
    capi.grlb_batch_step(b, 6)
    assert np.array_equal(capi.grlb_save(doms[1].h)[32:], before)
    assert doms[1].steps == 0 and doms[0].steps == 6 and doms[2].steps == 6
    capi.grlb_batch_set_active(b, None)
    capi.grlb_batch_step(b, 4)
    assert doms[1].steps == 4 and doms[0].steps == 10
    assert np.array_equal(capi.grlb_save(doms[0].h)[32:], batched_alone(cases[0], 10, schedule=schedule))
    capi.grlb_batch_destroy(b)


def test_large_domains_run_the_single_domain_sweep_inside_a_batch():
    """A domain of at least solo_min_cells cells is advanced by the kernel grlb_step runs:
    bitwise equal to the solo run; the small domains beside it go through the table."""
    big = inputs.tgv3d(40)          # 64000 cells
    small = mixed_cases()[2:4]
    cases = [big] + small
    doms = []
    for c in cases:
        d = capi.Domain(c.params)
        d.init(c.rho, c.u, c.p)
        doms.append(d)
    b = capi.grlb_batch_create([d.h for d in doms], use_graph=1, solo_min_cells=50000,
                               schedule=capi.SCHED_TABLE_CONST)
    capi.grlb_batch_step(b, 7)
    capi.grlb_batch_step(b, 6)
    _, raw_ref = solo(big, 13)
    assert np.array_equal(capi.grlb_save(doms[0].h)[32:], raw_ref)
    for c, d in zip(small, doms[1:]):
        assert d.steps == 13
        assert np.array_equal(capi.grlb_save(d.h)[32:], batched_alone(c, 13))
    capi.grlb_batch_destroy(b)


@pytest.mark.parametrize("schedule", TABLES)
@pytest.mark.parametrize("tile", [1, 32, 64, 128])
def test_every_tile_shape_gives_the_same_result(tile, schedule):
    """Linear tiles (1) and x-tiles of every width: bitwise the same batched result."""
    cases = mixed_cases()
    ref = [batched_alone(c, 9, schedule=schedule) for c in cases]
    doms = []
    for c in cases:
        d = capi.Domain(c.params)
        d.init(c.rho, c.u, c.p)
        doms.append(d)
    b = capi.grlb_batch_create([d.h for d in doms], use_graph=1, schedule=schedule)
    capi.grlb_batch_set_tile_x(b, [tile] * len(doms))
    capi.grlb_batch_step(b, 9)
    for c, d, r in zip(cases, doms, ref):
        assert np.array_equal(capi.grlb_save(d.h)[32:], r), (c.params.name, tile)
    capi.grlb_batch_destroy(b)


TUBES = ("becker", "sod")


def oracle_gate(case, Q, R):
    """The oracle comparison of a domain: rel L-inf 1e-5 on smooth fields, rel L1 1e-4 on the
    tubes (FP32 storage); 1e-2 / 6e-2 for FP16 / BF16 storage (the bounds of their other
    multi-step oracle comparisons; their rounding is pinned one sweep at a time in
    test_gpu_storage.py)."""
    tube = case.params.name.startswith(TUBES)
    err = rel_l1(Q, R) if tube else rel_linf(Q, R)
    fields = [0, 1, 4] if tube else [0, 1, 2, 3, 4]
    tol = {inputs.STORE_F32: 1e-4 if tube else 1e-5, inputs.STORE_F16: 1e-2,
           inputs.STORE_BF16: 6e-2}[case.params.storage]
    return np.all(err[fields] <= tol), err


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_batched_domains_match_the_oracle(schedule):
    cases = mixed_cases()
    doms = []
    for c in cases:
        d = capi.Domain(c.params)
        d.init(c.rho, c.u, c.p)
        doms.append(d)
    b = capi.grlb_batch_create([d.h for d in doms], use_graph=1, schedule=schedule)
    capi.grlb_batch_step(b, 100)
    capi.grlb_batch_destroy(b)
    for c, d in zip(cases, doms):
        R = run_oracle(c, 100).conserved()
        ok, err = oracle_gate(c, d.conserved(), R)
        assert ok, (c.params.name, c.params.storage, err)
        d.close()


def test_batches_beyond_the_constant_record_slots_fall_back_to_the_tile_table():
    """The small domains' records go to a constant table of 160 slots shared by all batches;
    a batch that finds too few free slots runs the tile-table sweep (records in device memory)
    instead, and gives the same results bit for bit.  Slots come back when a batch is
    destroyed."""
    cases = [inputs.random_smooth(8, 4, 2, seed=s) for s in range(170)]
    doms = []
    for c in cases:
        d = capi.Domain(c.params)
        d.init(c.rho, c.u, c.p)
        doms.append(d)
    big = capi.grlb_batch_create([d.h for d in doms], use_graph=1,   # 170 > 160: tile table
                                 schedule=capi.SCHED_TABLE_CONST)
    capi.grlb_batch_step(big, 9)
    capi.grlb_batch_destroy(big)
    for c, d in zip(cases[:12], doms[:12]):
        ref = batched_alone(c, 9)                                    # constant-table records
        assert np.array_equal(capi.grlb_save(d.h)[32:], ref), c.params.name
    # many batches in turn reuse the slots (each must find its own records)
    for rnd in range(3):
        part = doms[rnd * 50:(rnd + 1) * 50]
        b = capi.grlb_batch_create([d.h for d in part], use_graph=1, schedule=capi.SCHED_TABLE_CONST)
        capi.grlb_batch_step(b, 2)
        capi.grlb_batch_destroy(b)
        assert all(d.steps == 11 for d in part)
    for d in doms:
        d.close()


def test_table_schedules_agree():
    """Records in the constant table or in device memory: the same updates bit for bit; each
    schedule bitwise reproducible."""
    cases = mixed_cases()
    res = {}
    for mode in (capi.SCHED_TABLE_CONST, capi.SCHED_TABLE, capi.SCHED_TABLE_CONST):
        doms = []
        for c in cases:
            d = capi.Domain(c.params)
            d.init(c.rho, c.u, c.p)
            doms.append(d)
        b = capi.grlb_batch_create([d.h for d in doms], use_graph=1, schedule=mode)
        capi.grlb_batch_step(b, 11)
        capi.grlb_batch_destroy(b)
        got = [d.conserved() for d in doms]
        if mode in res:
            assert all(np.array_equal(x, y) for x, y in zip(got, res[mode]))
        res[mode] = got
        for d in doms:
            d.close()
    for c, x, y in zip(cases, res[capi.SCHED_TABLE_CONST], res[capi.SCHED_TABLE]):
        assert np.array_equal(x, y), c.params.name
    with pytest.raises(capi.GrlbError):
        capi.grlb_batch_create([capi.Domain(cases[0].params).h], schedule=3)


def test_two_lanes_give_each_domain_its_solo_batched_result():
    """Constant-table schedule: with enough tiles (here ~2000) the small domains are split into
    lanes stepped on their own streams (two by default, three with max_lanes 8, two with 2);
    every domain's result is still bitwise what it is batched alone (one lane)."""
    om = inputs.becker_tied_omega(8.0)
    cases = [inputs.tgv3d(48, mach=0.8, re=100.0), inputs.tgv3d(44, mach=1.0, re=100.0),
             inputs.becker(2048, mach=2.5, cells_per_front=8, omega=om, cfl_max=0.1, ny=4, nz=4),
             inputs.becker(1500, mach=4.0, cells_per_front=8, omega=om, cfl_max=0.1, ny=4, nz=4),
             inputs.tgv3d(20, storage=inputs.STORE_F16)]
    doms = []
    for c in cases:
        d = capi.Domain(c.params)
        d.init(c.rho, c.u, c.p)
        doms.append(d)
    for max_lanes in (0, 8):
        for d, c in zip(doms, cases):
            d.init(c.rho, c.u, c.p)
        b = capi.grlb_batch_create([d.h for d in doms], use_graph=1, solo_min_cells=10 ** 6,
                                   schedule=capi.SCHED_TABLE_CONST, max_lanes=max_lanes)
        capi.grlb_batch_step(b, 5)
        capi.grlb_batch_step(b, 8)
        capi.grlb_batch_destroy(b)
        for c, d in zip(cases, doms):
            assert d.steps == 13
            assert np.array_equal(capi.grlb_save(d.h)[32:], batched_alone(c, 13)), (c.params.name, max_lanes)
    for d in doms:
        d.close()
    with pytest.raises(capi.GrlbError):
        capi.grlb_batch_create([capi.Domain(cases[0].params).h], max_lanes=9)


def test_concurrent_schedule_with_many_domains_and_one_buffer():
    """Concurrent schedule: 40 domains over 32 side streams, one of them with one-buffer
    streaming, each bitwise its grlb_step result; the batch stream sees all of it done."""
    torch = pytest.importorskip("torch")
    cases = [inputs.random_smooth(8 + s % 7, 5, 3 + s % 4, seed=s) for s in range(39)]
    one = inputs.tgv3d(24)
    one.params = one.params.replace(streaming=1)
    cases.append(one)
    stream = torch.cuda.Stream()
    doms = []
    for c in cases:
        d = capi.Domain(c.params, stream=stream.cuda_stream)
        d.init(c.rho, c.u, c.p)
        doms.append(d)
    b = capi.grlb_batch_create([d.h for d in doms])
    capi.grlb_batch_step(b, 21)
    capi.grlb_batch_step(b, 18)
    capi.grlb_batch_destroy(b)
    for c, d in zip(cases, doms):
        assert d.steps == 39
        _, raw = solo(c, 39)
        assert np.array_equal(capi.grlb_save(d.h)[32:], raw), c.params.name
        d.close()


@pytest.mark.parametrize("schedule", [capi.SCHED_CONCURRENT, capi.SCHED_TABLE_CONST])
def test_full_batched_configuration_sampled_cells(schedule):
    """The 64-domain batched configuration (inputs.batched_mix(0): 48 Becker tubes of 128-2048 x
    4 x 4 cells, shock Mach 1.5-5, and 16 Taylor-Green boxes of 32^3-96^3), batched as the
    batched leg of the benchmark runs it (concurrent single-domain sweeps with graph replays) and
    with the constant-record table kernel: after 20 batched steps, one batched step of sampled
    cells of every domain -- both tube ends of a row and 40 random cells each -- against the
    oracle's update of the probed pre-step populations (ghost equilibria past the tube ends),
    within 2e-6 of each field's largest population as at 256^3; the sensor fires in some of
    them."""
    from tests.common import oracle_update_cells
    cases = inputs.batched_mix(0)
    doms = [capi.Domain(c.params) for c in cases]
    for d, c in zip(doms, cases):
        d.init(c.rho, c.u, c.p)
    b = capi.grlb_batch_create([d.h for d in doms], use_graph=1, schedule=schedule)
    capi.grlb_batch_step(b, 20)
    rng = np.random.default_rng(5)
    picks, wants, fired = [], [], 0
    for d, c in zip(doms, cases):
        prm = c.params
        N = prm.ncells
        cells = np.unique(np.concatenate([rng.integers(0, N, 40), [0, prm.nx - 1, N - 1]])).astype(np.int64)
        want, chi = oracle_update_cells(prm, lambda cs: capi.grlb_read_cells(d.h, cs), cells)
        picks.append(cells)
        wants.append(want)
        fired += int((chi > 0).sum())
    capi.grlb_batch_step(b, 1)
    capi.grlb_batch_destroy(b)
    for d, c, cells, want in zip(doms, cases, picks, wants):
        got = capi.grlb_read_cells(d.h, cells)
        assert d.steps == 21
        for k in range(5):
            blk = slice(7 * k, 7 * k + 7)
            scale = max(np.abs(want[blk]).max(), 1e-12)
            assert np.abs(got[blk] - want[blk]).max() / scale < 2e-6, (c.params.name, k)
        d.close()
    assert fired > 0
