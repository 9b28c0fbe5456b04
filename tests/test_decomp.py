"""z-slab decomposition on the CPU (no GPU): the ghost-plane exchange rule, applied to the FP64
oracle's populations, reproduces the undivided run bitwise; two gloo ranks, each owning one
slab, exchange the ghost slices with the multi-device path's rank-level exchange
(decomp.ring_exchange over torch.distributed) and all-reduce the interior totals; one rank
closes the ring on itself."""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2609_16361_b300 import decomp, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_slab_sizes_and_fields():
    assert decomp.slab_sizes(10, 3) == [4, 3, 3]
    assert decomp.slab_starts([4, 3, 3]) == [0, 4, 7]
    c = inputs.random_smooth(6, 5, 10, seed=2)
    s = decomp.slab_case(c, 0, 4)
    assert s.params.nz == 6
    nxy = 30
    # ghost plane 0 is the whole domain's last plane (periodic wrap), plane 1 its first
    np.testing.assert_array_equal(s.rho[:nxy], c.rho[9 * nxy:])
    np.testing.assert_array_equal(s.rho[nxy:2 * nxy], c.rho[:nxy])
    np.testing.assert_array_equal(s.u[2][5 * nxy:], c.u[2][4 * nxy:5 * nxy])
    with pytest.raises(ValueError):
        decomp.slab_case(inputs.sod(64), 0, 1)


def oracle_slabs(case, sizes, steps):
    parts = [decomp.slab_case(case, z0, n) for z0, n in zip(decomp.slab_starts(sizes), sizes)]
    orcs = []
    for p in parts:
        o = oracle.Oracle(p.params)
        o.init_primitive(p.rho, p.u, p.p)
        orcs.append(o)
    nxy = case.params.nx * case.params.ny
    S = len(orcs)
    for _ in range(steps):
        for i in range(S):
            decomp.exchange_planes(orcs[i].f, orcs[(i + 1) % S].f, nxy)
        for o in orcs:
            o.step(1)
    return orcs


@pytest.mark.parametrize("sizes", [[7, 9], [3, 5, 4, 4]])
def test_oracle_slabs_reproduce_the_undivided_run_bitwise(sizes):
    c = inputs.random_smooth(12, 10, 16, seed=4)
    whole = oracle.Oracle(c.params)
    whole.init_primitive(c.rho, c.u, c.p)
    whole.step(12)
    orcs = oracle_slabs(c, sizes, 12)
    nx, ny = c.params.nx, c.params.ny
    Q = decomp.stitch(decomp.interior(o.conserved_lattice(), nx, ny) for o in orcs)
    assert np.array_equal(Q, whole.conserved_lattice())


def test_without_exchange_the_slabs_diverge():
    """The exchange is what makes the slabs agree (each slab alone is its own periodic box)."""
    c = inputs.random_smooth(12, 10, 16, seed=4)
    whole = oracle.Oracle(c.params)
    whole.init_primitive(c.rho, c.u, c.p)
    whole.step(6)
    parts = [decomp.slab_case(c, 0, 8), decomp.slab_case(c, 8, 8)]
    Qs = []
    for p in parts:
        o = oracle.Oracle(p.params)
        o.init_primitive(p.rho, p.u, p.p)
        o.step(6)
        Qs.append(decomp.interior(o.conserved_lattice(), 12, 10))
    assert not np.array_equal(decomp.stitch(Qs), whole.conserved_lattice())


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle as orc
    from paper_2609_16361_b300 import decomp as dc
    from paper_2609_16361_b300 import inputs as inp
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        c = inp.random_smooth(10, 8, 12, seed=6)
        sizes = dc.slab_sizes(12, ws)
        z0 = dc.slab_starts(sizes)[rank]
        p = dc.slab_case(c, z0, sizes[rank])
        o = orc.Oracle(p.params)
        o.init_primitive(p.rho, p.u, p.p)
        nxy = 80
        for _ in range(8):
            # the rank-level exchange of the multi-device path (decomp.ring_exchange), on the
            # oracle slab's host slices instead of packed device buffers
            top = torch.from_numpy(np.ascontiguousarray(dc.top_slice(o.f, nxy)))
            bot = torch.from_numpy(np.ascontiguousarray(dc.bottom_slice(o.f, nxy)))
            from_down, from_up = dc.ring_exchange(top, bot, rank, ws)
            dc.put_bottom_ghost(o.f, nxy, from_down.numpy())
            dc.put_top_ghost(o.f, nxy, from_up.numpy())
            o.step(1)
        mine = dc.interior(o.conserved_lattice(), 10, 8)
        whole = orc.Oracle(c.params)
        whole.init_primitive(c.rho, c.u, c.p)
        whole.step(8)
        ref = whole.conserved_lattice()[:, z0 * nxy:(z0 + sizes[rank]) * nxy]
        totals = dc.allreduce_sum(mine.sum(axis=1))
        out.put((rank, bool(np.array_equal(mine, ref)), totals, whole.conserved_lattice().sum(axis=1)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_gloo_ranks_exchange_ghost_slices_and_allreduce_totals(ws):
    """Two ranks (the same peer above and below) and three (distinct peers)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + os.getpid() % 1000 + 10 * ws
    ps = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in ps:
        p.start()
    got = [q.get(timeout=180) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, same, totals, ref in got:
        assert same, rank
        np.testing.assert_allclose(totals, ref, rtol=1e-12, atol=1e-12)


def test_one_rank_closes_the_ring_on_itself():
    top, bot = object(), object()
    assert decomp.ring_exchange(top, bot, 0, 1) == (top, bot)
