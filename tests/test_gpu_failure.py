"""Failure detection, made on the host: a NaN written into a host field before the
initialisation (no GPU fault is involved; the kernels only carry the NaN forward).

- The diagnostic sweep counts the non-finite cells and grlb_diag_read returns GRLB_ENUMERIC
  with the record filled in; a clean state reads back normally.
- grlb_check_finite flags a non-finite state, in device memory and in page-locked host memory,
  for every storage type, and leaves the flag of a clean state untouched.
- The serving loop evicts a request whose state went non-finite and reports it as failed,
  while every other request's result stays bitwise what it is when served alone.
"""
import numpy as np
import pytest

from paper_2609_16361_b300 import capi, inputs, serve

pytestmark = pytest.mark.gpu

STORAGES = [inputs.STORE_F32, inputs.STORE_F16, inputs.STORE_BF16]


def poisoned(case, cell=37):
    rho = case.rho.copy()
    rho[cell] = np.nan
    return rho


@pytest.mark.parametrize("storage", STORAGES)
def test_diagnostics_report_a_nan_and_return_enumeric(storage):
    c = inputs.random_smooth(24, 20, 6, seed=2, storage=storage)
    bad = capi.Domain(c.params)
    bad.init(poisoned(c), c.u, c.p)
    bad.step(3)
    bad.step_diag()
    with pytest.raises(capi.GrlbError) as e:
        bad.diag()
    assert e.value.status == capi.GRLB_ENUMERIC
    g = bad.diag(allow_nonfinite=True)
    # the NaN spreads one cell per step along each axis: after 4 sweeps a diamond of cells
    assert 1 < g["n_nan"] < c.params.ncells and g["step"] == 4
    good = capi.Domain(c.params)
    good.init(c.rho, c.u, c.p)
    good.step(3)
    good.step_diag()
    assert good.diag()["n_nan"] == 0
    bad.close()
    good.close()


@pytest.mark.parametrize("storage", STORAGES)
def test_check_finite_flags_only_a_nonfinite_state(storage):
    torch = pytest.importorskip("torch")
    c = inputs.random_smooth(40, 21, 7, seed=5, storage=storage)  # ragged: partial last brick
    dev_flags = torch.zeros(2, dtype=torch.int32, device="cuda")
    host_flags = torch.zeros(2, dtype=torch.int32, pin_memory=True)
    for slot, rho in ((0, c.rho), (1, poisoned(c, cell=5000))):
        d = capi.Domain(c.params)
        d.init(rho, c.u, c.p)
        d.step(2)
        capi.grlb_check_finite(d.h, dev_flags.data_ptr() + 4 * slot)
        capi.grlb_check_finite(d.h, host_flags.data_ptr() + 4 * slot)
        torch.cuda.synchronize()
        d.close()
    assert dev_flags.cpu().tolist() == [0, 1]
    assert host_flags.tolist() == [0, 1]


def test_server_evicts_a_nonfinite_request_and_leaves_the_others_unchanged():
    trace = inputs.serving_trace(seed=3, n_requests=6, rate=200.0, tgv_range=(12, 20),
                                 steps_range=(60, 130))
    victim = max(trace, key=lambda r: r.steps)
    victim.case.rho = poisoned(victim.case, cell=victim.case.params.ncells // 2)
    # lookahead=1: the host waits for each chunk before enqueueing the next but one, so the
    # check of the victim's first chunk is read long before the victim could finish
    srv = serve.Server(chunk=16)
    res = srv.run(trace, realtime=False, lookahead=1)
    assert srv.evicted == 1
    # with chunks far ahead of the GPU the victim may finish before its flag is read: then the
    # readback reports it
    ahead = serve.Server(chunk=16).run(trace, realtime=False)
    assert [x.status for x in ahead] == [x.status for x in res]
    for r, x in zip(trace, res):
        if r is victim:
            assert x.status == "nonfinite" and x.digest == ""
            continue
        assert x.status == "ok"
        alone = serve.Server(chunk=16).run([r], realtime=False)[0]
        assert x.digest == alone.digest, f"request {r.rid} changed by the failing neighbour"
    assert serve.summarize(res)["failed"] == 1
