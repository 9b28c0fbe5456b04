"""Host-side logic of the batching and serving layers, without a GPU: the tile autotuner's size
classes, plans and table files, the server's per-request parameters and latency summary, and
the seeded workload generators (batched mix, serving trace) both run on."""
import math

import numpy as np
import pytest

from paper_2609_16361_b300 import autotune, inputs, serve


@pytest.mark.parametrize("shape,key", [((100, 4, 4), "nx128-tube"), ((32, 32, 32), "nx32-box"),
                                       ((2048, 4, 4), "nx4096-tube"), ((600, 8, 8), "nx4096-tube"),
                                       ((64, 9, 8), "nx64-box"), ((513, 1, 1), "nx4096-tube"),
                                       ((512, 16, 16), "nx512-box")])
def test_size_class_buckets(shape, key):
    """nx buckets <= 32, <= 64, <= 128, <= 512, larger; a tube has a cross-section of at most
    64 cells."""
    assert autotune.size_class(inputs.uniform(*shape).params) == key


def test_plan_uses_the_table_and_defaults_elsewhere(tmp_path):
    cases = [inputs.uniform(100, 4, 4), inputs.uniform(32, 32, 32), inputs.uniform(120, 2, 2)]
    table = {"nx128-tube": {"tile_x": 64, "mlups": {"1": 1.0, "64": 2.0}}}
    assert autotune.plan(cases, table) == [64, 0, 64]
    path = tmp_path / "sub" / "tune.json"
    autotune.save(table, str(path))
    assert autotune.load(str(path)) == table
    assert autotune.plan(cases, {}) == [0, 0, 0]


class _Req:
    def __init__(self, case):
        self.case = case


def test_request_params_one_buffer_only_for_large_requests():
    small, large = inputs.uniform(16, 4, 4), inputs.uniform(64, 64, 64)
    for one_buffer in (False, True):
        assert serve.request_params(_Req(small), 262144, one_buffer).streaming == 0
    assert serve.request_params(_Req(large), 262144, False).streaming == 0
    assert serve.request_params(_Req(large), 262144, True).streaming == 1
    # the request's own parameters are not modified
    assert large.params.streaming == 0


def test_summarize_latencies_and_rates():
    rs = []
    for i, (arr, fin) in enumerate([(0.0, 1.0), (0.5, 1.5), (1.0, 4.0), (2.0, 2.5)]):
        r = serve.Result(i, "sod", steps=100, cells=1000, arrival=arr)
        r.finished = fin
        rs.append(r)
    s = serve.summarize(rs)
    lat = np.array([1.0, 1.0, 3.0, 0.5])
    assert s["solves"] == 4
    assert s["span_s"] == pytest.approx(4.0)          # last finish - first arrival
    assert s["solves_per_s"] == pytest.approx(1.0)
    assert s["p50_latency_s"] == pytest.approx(np.percentile(lat, 50))
    assert s["p99_latency_s"] == pytest.approx(np.percentile(lat, 99))
    assert s["mean_latency_s"] == pytest.approx(1.375)
    assert s["mlups"] == pytest.approx(4 * 1000 * 100 / 4.0 / 1e6)
    assert serve.summarize(rs, t_span=8.0)["solves_per_s"] == pytest.approx(0.5)


def test_batched_mix_is_seeded_and_within_its_ranges():
    a = inputs.batched_mix(0, n_becker=6, n_tgv=2)
    b = inputs.batched_mix(0, n_becker=6, n_tgv=2)
    c = inputs.batched_mix(1, n_becker=6, n_tgv=2)
    shape = lambda m: [(x.params.nx, x.params.ny, x.params.nz) for x in m]
    assert shape(a) == shape(b) and shape(a) != shape(c)
    for x in a[:6]:
        assert 128 <= x.params.nx <= 2048 and (x.params.ny, x.params.nz) == (4, 4)
        assert x.params.bc == inputs.BC_X_DIRICHLET_EQ
    for x in a[6:]:
        assert 32 <= x.params.nx <= 96 and x.params.nx == x.params.ny == x.params.nz
        assert x.params.bc == inputs.BC_PERIODIC
    assert np.array_equal(a[0].rho, b[0].rho)


def test_serving_trace_is_seeded_poisson_and_within_its_ranges():
    kw = dict(n_requests=60, rate=20.0, tgv_range=(16, 20), steps_range=(10, 20))
    t1 = inputs.serving_trace(0, **kw)
    t2 = inputs.serving_trace(0, **kw)
    assert [(r.arrival, r.kind, r.steps, r.storage) for r in t1] == \
           [(r.arrival, r.kind, r.steps, r.storage) for r in t2]
    arr = np.array([r.arrival for r in t1])
    assert np.all(np.diff(arr) > 0) and arr[0] > 0
    # mean inter-arrival 1/rate: 60 exponential gaps, within 4 standard errors
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - 1 / 20.0) < 4 * (1 / 20.0) / math.sqrt(len(gaps))
    assert {r.kind for r in t1} == {"sod", "becker", "tgv"}
    assert {r.storage for r in t1} == {inputs.STORE_F16, inputs.STORE_F32}
    for r in t1:
        assert 10 <= r.steps <= 20 and r.case.params.storage == r.storage
        if r.kind == "tgv":
            assert 16 <= r.case.params.nx <= 20
        elif r.kind == "sod":
            assert 400 <= r.case.params.nx <= 4000
        else:
            assert 128 <= r.case.params.nx <= 2048
