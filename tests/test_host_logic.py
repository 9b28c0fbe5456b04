"""Host-side logic without a GPU: the tile autotuner's size classes, plans and table files, the
server's per-request parameters and latency summary, the seeded workload generators (batched
mix, serving trace) both run on, and the test suite's reader of the checkpoint format."""
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


@pytest.mark.parametrize("storage", [inputs.STORE_F32, inputs.STORE_F16, inputs.STORE_BF16])
def test_checkpoint_decode_reads_the_documented_brick_layout(storage):
    """decode_populations (used by the population-level GPU parity tests) against a checkpoint
    body written here from the header's description: ceil(N / 128) bricks of 35 rows x 128
    cells, element (c // 128) 4480 + 128 q + c % 128, deviations from the reference
    equilibrium, FP16 deviations times 2^8 / M_k rounded to a power of two."""
    from tests.common import CI, WI, decode_populations
    prm = inputs.uniform(10, 7, 3, storage=storage).params  # N = 210: two bricks, ragged
    N = 210
    s = prm.dt / prm.dx
    p_ref = prm.ref_p * s * s
    E_ref = p_ref / (prm.gamma - 1)
    rng = np.random.default_rng(3)
    dev = rng.normal(size=(35, N)) * 1e-2  # deviations d_{k,i}
    if storage == inputs.STORE_F16:
        c_ref = math.sqrt(prm.gamma * p_ref / prm.ref_rho)
        M = [prm.ref_rho, prm.ref_rho * c_ref, prm.ref_rho * c_ref, prm.ref_rho * c_ref, E_ref]
        enc = [2.0 ** (8 - round(math.log2(m))) for m in M]
    else:
        enc = [1.0] * 5
    stored = np.stack([dev[q] * enc[q // 7] for q in range(35)])
    dtype = {inputs.STORE_F32: np.float32, inputs.STORE_F16: np.float16}.get(storage)
    if storage == inputs.STORE_BF16:  # truncate FP32 to its top 16 bits (bfloat16)
        bits = (stored.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
        stored_exact = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        body_vals = bits
    else:
        body_vals = stored.astype(dtype)
        stored_exact = body_vals.astype(np.float64)
    nb = 2
    body = np.zeros((nb, 35, 128), dtype=body_vals.dtype)
    for c in range(N):
        body[c // 128, :, c % 128] = body_vals[:, c]
    raw = np.concatenate([np.zeros(32, np.uint8), body.reshape(-1).view(np.uint8)])
    f = decode_populations(raw, prm)
    Qref = [prm.ref_rho, 0, 0, 0, E_ref]
    for q in range(35):
        k, i = divmod(q, 7)
        Jref = np.zeros(3)
        if 1 <= k <= 3:
            Jref[k - 1] = p_ref
        shift = WI[i] * (Qref[k] + 4.0 * CI[i] @ Jref)
        np.testing.assert_allclose(f[q], stored_exact[q] / enc[k] + shift, rtol=0, atol=1e-15)
    cells = np.array([0, 127, 128, 209])
    np.testing.assert_array_equal(decode_populations(raw, prm, cells=cells), f[:, cells])


def test_bf16_rounding_helper_matches_torch():
    """The storage test's own bfloat16 rounding (nearest, ties to even) against torch's
    conversion, on the CPU."""
    torch = pytest.importorskip("torch")
    from tests.test_gpu_storage import bf16_round
    x = np.random.default_rng(1).normal(size=20000) * np.logspace(-3, 3, 20000)
    x = np.concatenate([x, [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(bf16_round(x), ref)


def test_device_taylor_green_fields_equal_the_host_generator():
    """inputs.tgv3d_device (fields built plane by plane as torch tensors, here on the CPU)
    gives tgv3d's parameters and, bit for bit, its fields."""
    torch = pytest.importorskip("torch")
    for n, kw in ((8, {}), (12, dict(mach=0.8, storage=inputs.STORE_F16))):
        c = inputs.tgv3d(n, **kw)
        prm, rho, u, p = inputs.tgv3d_device(n, device="cpu", **kw)
        assert prm == c.params
        assert np.array_equal(rho.numpy(), c.rho) and np.array_equal(u.numpy(), c.u)
        assert np.array_equal(p.numpy(), c.p)


def test_per_cell_oracle_update_equals_the_oracle_sweep():
    """The per-cell update the sampled-cell parity tests use (tests.common.oracle_update_cells:
    pull sources by periodic wrap, ghost equilibria past the ends of a Dirichlet tube) gives
    bit for bit the oracle's own sweep, for every cell of two tubes and a periodic box."""
    import oracle
    from tests.common import oracle_update_cells
    for c in (inputs.sod(64), inputs.becker(128, ny=4, nz=4), inputs.random_smooth(12, 5, 4, seed=2)):
        o = oracle.Oracle(c.params)
        o.init_primitive(c.rho, c.u, c.p)
        o.step(3)
        pre = o.f.copy()
        o.step(1)
        cells = np.arange(c.params.ncells)
        want, _ = oracle_update_cells(c.params, lambda cs: pre[:, cs], cells)
        assert np.array_equal(want, o.f[:, cells]), c.params.name


def test_counter_records_are_keyed_to_code_not_comments():
    """bench.py attaches an ncu counter record to its line only while the kernel sources' code
    is the code the counters were taken on: comment and blank-line edits keep the key, any code
    change (an operand, a launch bound) drops it."""
    import bench
    base = "// header\n__global__ void k(float* a) {  // one thread per element\n    a[0] = 1.0f;\n}\n"
    src = {"a.cu": base}
    key = bench.kernel_source_sha(["a.cu"], read=src.get)
    src["a.cu"] = "// header, reworded\n\n__global__ void k(float* a) {\n    a[0] = 1.0f;   // store\n}\n"
    assert bench.kernel_source_sha(["a.cu"], read=src.get) == key
    for edit in ("a[0] = 2.0f;", "a[1] = 1.0f;"):
        src["a.cu"] = base.replace("a[0] = 1.0f;", edit)
        assert bench.kernel_source_sha(["a.cu"], read=src.get) != key
    # a file boundary is part of the key: the same lines split differently between files differ
    two = {"a.cu": "int x;\nint y;", "b.cu": "int z;"}
    moved = {"a.cu": "int x;", "b.cu": "int y;\nint z;"}
    assert bench.kernel_source_sha(["a.cu", "b.cu"], read=two.get) != bench.kernel_source_sha(["a.cu", "b.cu"], read=moved.get)


def test_l2_prefetch_addresses_stay_inside_the_state_buffer():
    """The sweeps' bulk L2 prefetches (not seen by the bounds-checked build, which issues none)
    replayed on the host with the kernels' index arithmetic for every CTA of many launches:
    each prefetched range is one whole brick (20 moment rows x 128 FP32 values, or 35
    population rows x 128 16-bit values), starts on a 16-byte boundary and lies inside the
    buffer.  Moment sweep: lane 0 of each tile row whose x starts a brick, planes z + 1 (first
    plane of a chunk) and z + 2 below nz; 16-bit sweep: the same lane, plane z + 2 below nz;
    both only when nx is a multiple of 128 and nx ny <= 256^2."""
    BR, NM, NP = 128, 20, 35
    for nx in (128, 256, 384, 512):
        for ny in (1, 3, 4, 8, 37):
            for nz in (1, 2, 3, 5, 8):
                N = nx * ny * nz
                if nx % BR or nx * ny > 256 * 256:
                    continue
                nbricks = -(-N // BR)
                for bx, by in ((32, 4), (64, 2), (128, 1)):
                    lz = min(nz, 4)
                    for gx in range(-(-nx // bx)):
                        x = gx * bx                      # lane threadIdx.x == 0
                        if x % BR:
                            continue
                        for gy in range(-(-ny // by)):
                            for ty in range(by):
                                y = gy * by + ty
                                if y >= ny:
                                    continue
                                for gz in range(-(-nz // lz)):       # moment column kernel
                                    zb, ze = gz * lz, min(gz * lz + lz, nz)
                                    for z in range(zb, ze):
                                        for zz in range(z + 1 if z == zb else z + 2, min(z + 2, nz - 1) + 1):
                                            c = (y + ny * zz) * nx + x
                                            assert c % BR == 0 and c < N
                                            start = (c // BR) * NM * BR * 4          # bytes
                                            assert start % 16 == 0 and (NM * BR * 4) % 16 == 0
                                            assert start + NM * BR * 4 <= nbricks * NM * BR * 4
                                for z in range(nz):                  # 16-bit population sweep
                                    if z + 2 < nz:
                                        c = (y + ny * (z + 2)) * nx + x
                                        start = (c // BR) * NP * BR * 2
                                        assert c % BR == 0 and start % 16 == 0 and (NP * BR * 2) % 16 == 0
                                        assert start + NP * BR * 2 <= nbricks * NP * BR * 2
