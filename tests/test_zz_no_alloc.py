"""The allocation-free diagnostic sweep (grlb_step_diag_noalloc) against grlb_step_diag.

grlb_step_diag_noalloc serves callers that cannot call cudaMalloc (a host whose memory manager
reserved the device memory up front, or a time-critical loop that cannot take cudaMalloc's
implicit synchronisation): it keeps its block partials in a static device array instead.  The
test plays such a caller: the population buffers and the result record are its own device
memory, and two calls in a row must give what the allocating entry point gives.  It lives in
its own file, collected last, and works alone in a fresh process or after the other tests.
"""
import numpy as np
import pytest

from paper_2609_16361_b300 import capi, inputs

pytestmark = pytest.mark.gpu

HDR = 32  # bytes of the grlb_save header before the populations


CASES = {
    # name: (grid, storage, collision)
    "tgv32_f32_rlb": ("tgv32", inputs.STORE_F32, inputs.COLL_RLB_SENSOR),
    "ragged_f32_rlb": ("ragged", inputs.STORE_F32, inputs.COLL_RLB_SENSOR),
    "tgv32_f16_rlb": ("tgv32", inputs.STORE_F16, inputs.COLL_RLB_SENSOR),
    "tgv32_bf16_rlb": ("tgv32", inputs.STORE_BF16, inputs.COLL_RLB_SENSOR),
    "ragged_f32_bgk": ("ragged", inputs.STORE_F32, inputs.COLL_BGK),
}


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_diag_sweep_matches_allocating_entry_point_twice(name):
    """tgv32: 256 whole cell bricks; ragged: 40 x 21 x 7 = 5880 cells, 46 bricks, the last one
    partly used (the caller's buffers hold whole bricks; the unused cells are never written,
    so the output buffer starts zeroed like the library's own).  Both entry points run the same
    kernel on the same record with the same launch shape, so populations and the diagnostic
    record must agree bit for bit, for every storage type and both collisions."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    grid, storage, collision = CASES[name]
    c = inputs.tgv3d(32) if grid == "tgv32" else inputs.random_smooth(40, 21, 7, seed=9)
    prm = c.params.replace(storage=storage, collision=collision)
    N = prm.ncells
    esize = 4 if storage == inputs.STORE_F32 else 2
    d = capi.Domain(prm)
    d.init(c.rho, c.u, c.p)
    d.step(7)
    torch.cuda.synchronize()
    state = capi.grlb_save(d.h)[HDR:]
    assert state.size == 35 * 128 * (-(-N // 128)) * esize
    f_a = torch.from_numpy(state.copy()).cuda()
    f_b = torch.zeros_like(f_a)
    diag = torch.zeros(13, dtype=torch.float64, device="cuda")
    Qref = np.array([prm.ref_rho, 0, 0, 0, prm.ref_p * (prm.dt / prm.dx) ** 2 / (prm.gamma - 1)])
    src, dst = f_a, f_b
    for call in range(2):
        diag.fill_(-1.0)
        torch.cuda.synchronize()
        capi.grlb_step_diag_noalloc(prm, src.data_ptr(), dst.data_ptr(), diag.data_ptr(), None)
        torch.cuda.synchronize()
        d.step_diag()
        want = d.diag()
        ref_pops = capi.grlb_save(d.h)[HDR:]
        got_pops = dst.cpu().numpy()
        assert np.array_equal(got_pops, ref_pops), f"call {call}: populations differ"
        g = diag.cpu().numpy()
        np.testing.assert_allclose(N * Qref + g[:5], want["totals"], rtol=1e-15, atol=0)
        assert list(g[5:10]) == [want["ke"], want["eps_s"], want["eps_d"], want["rho_min"],
                                 want["p_min"]], f"call {call}: diagnostic sums"
        assert [int(v) for v in g[10:13]] == [want["n_floor"], want["n_nan"], want["n_sensor"]]
        src, dst = dst, src
    d.close()


def test_noalloc_rejects_domains_beyond_the_static_scratch():
    big = inputs.tgv3d(256).params  # 131072 CTAs of 128 cells
    with pytest.raises(capi.GrlbError, match="static scratch"):
        capi.grlb_step_diag_noalloc(big, 1, 2, 3, None)
