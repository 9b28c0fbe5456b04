"""z-slab decomposition on one GPU (grlb_halo_exchange_z): the interior of the slabs evolves
bitwise as the undivided domain, for uneven slabs, ragged CTA tiles, FP16 storage and the
Chapman-Enskog start; interior totals add up to the whole domain's.  The multi-device form
(grlb_halo_pack_z / grlb_halo_unpack_z around a transfer of device buffers) gives the same:
one rank whose ring closes on itself (decomp.SlabRank, world 1), and slabs that swap their packed
slices through device buffers as ranks on different devices would."""
import dataclasses

import numpy as np
import pytest

from paper_2609_16361_b300 import capi, decomp, inputs

pytestmark = pytest.mark.gpu


def whole_run(case, steps, ce=None):
    d = capi.Domain(case.params.replace(streaming=0))
    d.init(case.rho, case.u, case.p, ce_init=ce)
    d.step(steps)
    Q = d.conserved()
    d.close()
    return Q


def slab_run(case, sizes, steps, ce=None):
    s = decomp.SlabSet(case, sizes)
    s.init(ce_init=ce)
    s.step(steps)
    Q = s.conserved()
    tot = s.interior_totals()
    s.close()
    return Q, tot


@pytest.mark.parametrize("case,sizes,steps", [
    (lambda: inputs.tgv3d(32), [16, 16], 40),
    (lambda: inputs.random_smooth(40, 21, 24, seed=5), [5, 9, 10], 30),
    (lambda: inputs.tgv3d(32, storage=inputs.STORE_F16), [12, 20], 30),
    (lambda: inputs.random_smooth(32, 32, 32, seed=8, collision=inputs.COLL_BGK), [8, 8, 8, 8], 25),
])
def test_slabs_bitwise_equal_the_undivided_run(case, sizes, steps):
    c = case()
    Qw = whole_run(c, steps)
    Qs, tot = slab_run(c, sizes, steps)
    assert np.array_equal(Qs, Qw)
    np.testing.assert_allclose(np.sum(tot, axis=0), Qw.sum(axis=1), rtol=1e-12)


def test_slabs_with_chapman_enskog_start():
    c = inputs.tgv3d(32, mach=0.5, re=100.0, fmu=0.001)
    assert np.array_equal(slab_run(c, [10, 22], 20, ce=True)[0], whole_run(c, 20, ce=True))


def test_exchange_rejects_unsuitable_slabs():
    c = inputs.random_smooth(16, 16, 16, seed=1)
    a = capi.Domain(c.params)
    b = capi.Domain(c.params.replace(streaming=1))
    e = capi.Domain(c.params.replace(nx=8))
    for x, y in ((a, b), (a, e)):
        with pytest.raises(capi.GrlbError):
            capi.grlb_halo_exchange_z(x.h, y.h)
    for d in (a, b, e):
        d.close()


@pytest.mark.parametrize("storage", [inputs.STORE_F32, inputs.STORE_F16])
def test_one_rank_ring_equals_the_periodic_domain(storage):
    c = inputs.tgv3d(32, storage=storage)
    r = decomp.SlabRank(c, 0, 1)
    r.init()
    r.step(25)
    assert np.array_equal(r.conserved_interior(), whole_run(c, 25))
    r.close()


def test_packed_slices_between_slabs_equal_the_undivided_run():
    """Three slabs exchange through packed device buffers (the transfer a multi-rank run makes
    with NCCL is a plain copy here): bitwise the undivided run."""
    torch = pytest.importorskip("torch")
    c = inputs.random_smooth(40, 21, 24, seed=5)
    sizes = [7, 9, 8]
    parts = [decomp.slab_case(c, z0, n) for z0, n in zip(decomp.slab_starts(sizes), sizes)]
    doms = [capi.Domain(p.params) for p in parts]
    for d, p in zip(doms, parts):
        d.init(p.rho, p.u, p.p)
    nxy = 40 * 21
    bufs = [(torch.empty((5, nxy), device="cuda"), torch.empty((5, nxy), device="cuda")) for _ in doms]
    recv = [(torch.empty((5, nxy), device="cuda"), torch.empty((5, nxy), device="cuda")) for _ in doms]
    S = len(doms)
    for _ in range(30):
        for d, (up, down) in zip(doms, bufs):
            capi.grlb_halo_pack_z(d.h, up.data_ptr(), down.data_ptr())
        torch.cuda.synchronize()
        for i in range(S):
            recv[i][0].copy_(bufs[(i - 1) % S][0])   # from below: the lower slab's top slice
            recv[i][1].copy_(bufs[(i + 1) % S][1])   # from above: the upper slab's bottom slice
        torch.cuda.synchronize()
        for d, (below, above) in zip(doms, recv):
            capi.grlb_halo_unpack_z(d.h, below.data_ptr(), above.data_ptr())
            d.step(1)
    Q = decomp.stitch(decomp.interior(d.conserved(), 40, 21) for d in doms)
    assert np.array_equal(Q, whole_run(c, 30))
    with pytest.raises(capi.GrlbError):
        capi.grlb_halo_pack_z(capi.Domain(inputs.sod(64).params).h, 1, 2)
    for d in doms:
        d.close()


def test_moment_slabs_bitwise_equal_the_undivided_moment_run():
    """Moment storage: the exchange carries Q_k / 8 and J*_k,z of the boundary planes (on one device
    and through packed buffers, one rank closing the ring on itself); the interior is bitwise
    the undivided moment run, which is bitwise the population run."""
    c = inputs.tgv3d(32)
    mc = dataclasses.replace(c, params=c.params.replace(streaming=2))
    want = whole_run(c, 30)
    d = capi.Domain(mc.params)
    d.init(c.rho, c.u, c.p)
    d.step(30)
    assert np.array_equal(d.conserved(), want)
    d.close()
    s = decomp.SlabSet(mc, [12, 20])
    s.init()
    s.step(30)
    assert np.array_equal(s.conserved(), want)
    s.close()
    r = decomp.SlabRank(mc, 0, 1)
    assert tuple(r.top.shape) == (10, 32 * 32)
    r.init()
    r.step(30)
    assert np.array_equal(r.conserved_interior(), want)
    r.close()
    a, b = capi.Domain(c.params), capi.Domain(mc.params.replace(nz=32))
    with pytest.raises(capi.GrlbError):  # slabs of different kinds
        capi.grlb_halo_exchange_z(a.h, b.h)
    a.close()
    b.close()
