"""Serving loop: continuous batching of simulation requests of different sizes, step counts
and storage types.  Each request's result is bitwise the same served alone and in the mix,
and bitwise the plain single-domain path's with the same storage (the batched kernels round
every operation as the single-domain sweep does: no compiler contraction in the sweep file).
Admission respects the HBM budget."""
import numpy as np
import pytest

from paper_2609_16361_b300 import capi, inputs, serve
from tests.common import run_oracle
from tests.test_gpu_batch import oracle_gate

pytestmark = pytest.mark.gpu


def small_trace(n=8, seed=3):
    return inputs.serving_trace(seed=seed, n_requests=n, rate=200.0, tgv_range=(12, 20),
                                steps_range=(20, 130))


def test_each_result_is_the_same_alone_and_in_the_mix():
    trace = small_trace()
    assert len({r.storage for r in trace}) == 2 and len({r.kind for r in trace}) >= 2
    mixed = serve.Server(chunk=16, keep_fields=True).run(trace, realtime=False)
    plain = serve.serial_plain(trace, realtime=False, keep_fields=True)
    for r, m, p in zip(trace, mixed, plain):
        alone = serve.Server(chunk=16).run([r], realtime=False)[0]
        assert m.rid == r.rid == alone.rid == p.rid
        assert m.digest == alone.digest, f"request {r.rid} ({r.kind}) differs in the mix"
        assert m.status == alone.status == p.status == "ok"
        assert np.array_equal(m.fields, p.fields), (r.rid, r.kind, r.storage)


def test_shortest_remaining_work_first_keeps_results_unchanged():
    trace = small_trace(n=6, seed=7)
    a = serve.Server(chunk=8, large_cells=2000, srpt=True).run(trace, realtime=False)
    b = serve.Server(chunk=8, large_cells=2000, srpt=False).run(trace, realtime=False)
    assert [x.digest for x in a] == [y.digest for y in b]


def test_admission_respects_a_shrunken_budget():
    trace = small_trace(n=6, seed=4)
    sizes = [capi.grlb_bytes_for(r.case.params) for r in trace]
    budget = 1.5 * max(sizes)
    srv = serve.Server(hbm_budget=budget, chunk=10)
    res = srv.run(trace, realtime=False)
    assert len(res) == len(trace) and all(r.digest for r in res)
    assert srv.peak_bytes <= budget
    ref = serve.Server(chunk=10).run(trace, realtime=False)
    assert [a.digest for a in res] == [b.digest for b in ref]


def test_request_larger_than_budget_is_refused():
    trace = small_trace(n=1, seed=5)
    with pytest.raises(capi.GrlbError):
        serve.Server(hbm_budget=1000).run(trace, realtime=False)


def test_one_buffer_large_requests():
    """Large requests with one population buffer: half their device memory, results within
    FP32 rounding of the two-buffer ones (the same collisions), small requests unchanged
    bitwise, and still independent of the mix."""
    trace = small_trace(n=8, seed=11)
    large = 3000
    big = [r for r in trace if r.case.params.ncells >= large]
    assert big and len(big) < len(trace)
    for r in big:
        one = capi.grlb_bytes_for(serve.request_params(r, large, True))
        two = capi.grlb_bytes_for(r.case.params)
        assert one < 0.6 * two
    a = serve.Server(chunk=12, large_cells=large, one_buffer_large=True, keep_fields=True).run(trace, realtime=False)
    b = serve.Server(chunk=12, large_cells=large, keep_fields=True).run(trace, realtime=False)
    for r, x, y in zip(trace, a, b):
        if r.case.params.ncells < large:
            assert x.digest == y.digest
        else:
            assert np.array_equal(x.fields, y.fields), r.rid
    r0 = big[0]
    alone = serve.Server(chunk=12, large_cells=large, one_buffer_large=True).run([r0], realtime=False)[0]
    assert alone.digest == a[trace.index(r0)].digest


def test_served_results_match_the_oracle():
    """Every request of the mixed trace against the FP64 oracle run of its own case: FP32
    requests at rel L-inf 1e-5 (Taylor-Green boxes) / rel L1 1e-4 (Sod and Becker tubes), FP16
    requests within 1e-2."""
    trace = small_trace()
    res = serve.Server(chunk=16, keep_fields=True).run(trace, realtime=False)
    assert sum(r.storage == inputs.STORE_F32 for r in trace) >= 3
    for r, x in zip(trace, res):
        R = run_oracle(r.case, r.steps).conserved()
        ok, err = oracle_gate(r.case, x.fields, R)
        assert ok, (r.rid, r.kind, r.storage, err)


def test_served_moment_requests_equal_their_population_runs():
    """With moments, the FP32 requests keep their state as moments: every result bitwise the
    population server's (and the serial baseline's in the same state)."""
    trace = small_trace(n=8, seed=5)
    assert any(r.storage == inputs.STORE_F32 for r in trace)
    a = serve.Server(chunk=16, keep_fields=True).run(trace, realtime=False)
    b = serve.Server(chunk=16, keep_fields=True, moments=True).run(trace, realtime=False)
    c = serve.serial_plain(trace, realtime=False, keep_fields=True, moments=True)
    for r, x, y, z in zip(trace, a, b, c):
        assert x.status == y.status == "ok"
        assert x.digest == y.digest, (r.rid, r.kind, r.storage)
        assert np.array_equal(z.fields, y.fields), (r.rid, r.kind, r.storage)
