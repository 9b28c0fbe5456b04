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


@pytest.mark.parametrize("case", ["tgv32", "ragged"])
def test_noalloc_diag_sweep_matches_allocating_entry_point_twice(case):
    """tgv32: 256 whole cell bricks; ragged: 40 x 21 x 7 = 5880 cells, 46 bricks, the last one
    partly used (the caller's buffers hold whole bricks; the unused cells are never written,
    so the output buffer starts zeroed like the library's own)."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    c = inputs.tgv3d(32) if case == "tgv32" else inputs.random_smooth(40, 21, 7, seed=9)
    prm = c.params
    N = prm.ncells
    d = capi.Domain(prm)
    d.init(c.rho, c.u, c.p)
    d.step(7)
    torch.cuda.synchronize()
    state = capi.grlb_save(d.h)[HDR:]
    assert state.size == 35 * 128 * (-(-N // 128)) * 4
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
        ref_pops = capi.grlb_save(d.h)[HDR:].view(np.float32)
        got_pops = dst.cpu().numpy().view(np.float32)
        scale = np.abs(ref_pops).max()
        assert np.abs(got_pops - ref_pops).max() <= 1e-5 * scale, f"call {call}: populations"
        g = diag.cpu().numpy()
        np.testing.assert_allclose(N * Qref + g[:5], want["totals"], rtol=1e-6,
                                   atol=1e-6 * N * prm.ref_rho)
        np.testing.assert_allclose(g[5:8], [want["ke"], want["eps_s"], want["eps_d"]], rtol=1e-5)
        np.testing.assert_allclose(g[8:10], [want["rho_min"], want["p_min"]], rtol=1e-6)
        assert [int(v) for v in g[10:13]] == [want["n_floor"], want["n_nan"], want["n_sensor"]]
        src, dst = dst, src
    d.close()


def test_noalloc_rejects_domains_beyond_the_static_scratch():
    big = inputs.tgv3d(256).params  # 131072 CTAs of 128 cells
    with pytest.raises(capi.GrlbError, match="static scratch"):
        capi.grlb_step_diag_noalloc(big, 1, 2, 3, None)
