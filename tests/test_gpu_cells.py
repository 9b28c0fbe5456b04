"""Point probes (grlb_read_cells) and, through them, sampled-cell parity at the capacity sizes.

grlb_read_cells returns the post-collision populations f*_q of listed cells in FP64 lattice
units for every streaming pattern.  Pinned three ways: against the documented checkpoint format
decoded independently (two buffers, every storage type); one-buffer domains after odd steps
(values gathered from the neighbours and the outflow record) and even steps (swapped slots)
against the two-buffer run of the same steps, with a check that a wrong slot would show; and
the sum over links against grlb_read_conserved.  Then the capacity configurations -- 1024^3 with
FP16 populations and 768^3 with FP32, one population buffer each, the workload `bench.py
--workload capacity` times, and 1024^3 FP32 with the state as moments -- one sweep of sampled
cells against the oracle's update of the same cells from the probed pre-step populations of their
pull sources."""
import numpy as np
import pytest

from paper_2609_16361_b300 import capi, inputs
from tests.common import CI, decode_populations, oracle_update_cells
from tests.test_gpu_storage import spacing

pytestmark = pytest.mark.gpu


def run(case, steps, streaming=0):
    d = capi.Domain(case.params.replace(streaming=streaming))
    d.init(case.rho, case.u, case.p)
    d.step(steps)
    return d


@pytest.mark.parametrize("storage", [inputs.STORE_F32, inputs.STORE_F16, inputs.STORE_BF16])
def test_probes_equal_the_decoded_checkpoint(storage):
    c = inputs.random_smooth(40, 21, 7, seed=3, storage=storage)
    d = run(c, 3)
    N = c.params.ncells
    cells = np.array([0, 1, 39, 40, N // 2, N - 128, N - 1] + list(range(100, 5000, 37)))
    got = capi.grlb_read_cells(d.h, cells)
    want = decode_populations(capi.grlb_save(d.h), c.params, cells=cells)
    scale = np.abs(want).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - want) <= 1e-14 * scale)
    assert capi.grlb_read_cells(d.h, []).shape == (35, 0)
    for bad in ([-1], [N], [0, N + 5]):
        with pytest.raises(capi.GrlbError):
            capi.grlb_read_cells(d.h, bad)
    d.close()


@pytest.mark.parametrize("case", [lambda: inputs.tgv3d(16), lambda: inputs.sod(64),
                                  lambda: inputs.random_smooth(33, 5, 4, seed=1, collision=inputs.COLL_BGK)])
@pytest.mark.parametrize("steps", [1, 2, 3])
def test_one_buffer_probes_equal_the_two_buffer_run(case, steps):
    """Odd steps: f*_i(x) sits in slot i of x + c_i (the outflow record past the ends of a
    tube); even steps: in slot opp(i) of x.  The probes of the one-buffer run equal those of the
    two-buffer run bit for bit, for every cell including the tube ends (and a probe that read
    the opposite link would be off by far more than rounding)."""
    c = case()
    a, b = run(c, steps, 0), run(c, steps, 1)
    cells = np.arange(c.params.ncells)
    fa, fb = capi.grlb_read_cells(a.h, cells), capi.grlb_read_cells(b.h, cells)
    assert np.array_equal(fa, fb), steps
    # a probe that read the opposite link would be off by far more than the tolerance
    swap = np.abs(fa[[1, 3, 5]] - fa[[2, 4, 6]]).max() / np.abs(fa[0:7]).max()
    assert swap > 1e-3
    a.close()
    b.close()


@pytest.mark.parametrize("streaming", [0, 1])
def test_probe_sums_are_the_conserved_fields(streaming):
    c = inputs.tgv3d(12, storage=inputs.STORE_F16)
    d = run(c, 5, streaming)
    s = c.params.dt / c.params.dx
    f = capi.grlb_read_cells(d.h, np.arange(c.params.ncells))
    Q = np.stack([f[7 * k:7 * k + 7].sum(axis=0) for k in range(5)])
    R = d.conserved()
    R[1:4] *= s
    R[4] *= s * s
    for k in range(5):
        assert np.abs(Q[k] - R[k]).max() <= 1e-12 * np.abs(R[k]).max(), k
    d.close()


def stored_values(f, prm):
    """FP64 populations -> the 16-bit stored deviations they decode from (exact inverse of the
    decoding up to FP64 rounding), as (35, n) float64."""
    s = prm.dt / prm.dx
    p_ref = prm.ref_p * s * s
    E_ref = p_ref / (prm.gamma - 1)
    c_ref = np.sqrt(prm.gamma * p_ref / prm.ref_rho)
    M = [prm.ref_rho, prm.ref_rho * c_ref, prm.ref_rho * c_ref, prm.ref_rho * c_ref, E_ref]
    Qref = [prm.ref_rho, 0, 0, 0, E_ref]
    out = np.empty_like(f)
    for k in range(5):
        enc = 2.0 ** (8 - int(round(np.log2(M[k])))) if prm.storage == inputs.STORE_F16 else 1.0
        Jref = np.zeros(3)
        if 1 <= k <= 3:
            Jref[k - 1] = p_ref
        for i in range(7):
            out[7 * k + i] = (f[7 * k + i] - 0.125 * (2.0 if i == 0 else 1.0) * (Qref[k] + 4.0 * CI[i] @ Jref)) * enc
    return out


@pytest.mark.parametrize("n,storage", [(1024, inputs.STORE_F16), (768, inputs.STORE_F32)])
def test_capacity_sizes_sampled_cells(n, storage):
    """One population buffer at the capacity sizes (75 GB FP16 / 63 GB FP32 of populations),
    fields built on the device, Taylor-Green as in the headline workload: after 5 sweeps (odd:
    the gathered layout) one more sweep (even layout) of 2000 sampled cells -- among them the
    first and last cells and the ends of rows, planes and the last brick -- against the
    oracle's update of the probed pre-step populations.  FP32: within 2e-6 of each field's
    largest population (as at 256^3).  FP16: every stored value is the rounded oracle value up
    to one FP16 spacing plus 16 units of 2^-24 of the field's largest stored value (the bound
    of the one-sweep storage pin)."""
    torch = pytest.importorskip("torch")
    torch.cuda.empty_cache()
    capi.grlb_trim_pool()
    prm, rho, u, p = inputs.tgv3d_device(n, storage=storage)
    prm = prm.replace(streaming=1)
    d = capi.Domain(prm)
    capi.grlb_init_primitive_device(d.h, rho.data_ptr(), u.data_ptr(), p.data_ptr())
    torch.cuda.synchronize()
    del rho, u, p
    torch.cuda.empty_cache()
    d.step(5)
    N = prm.ncells
    rng = np.random.default_rng(11)
    edges = [0, 1, n - 1, n, n * n - 1, n * n, N - n, N - 128, N - 1]
    cells = np.unique(np.concatenate([rng.integers(0, N, 2000), edges])).astype(np.int64)
    want, _ = oracle_update_cells(prm, lambda cs: capi.grlb_read_cells(d.h, cs), cells)
    d.step(1)
    got = capi.grlb_read_cells(d.h, cells)
    d.close()
    if storage == inputs.STORE_F32:
        for k in range(5):
            blk = slice(7 * k, 7 * k + 7)
            scale = max(np.abs(want[blk]).max(), 1e-12)
            assert np.abs(got[blk] - want[blk]).max() / scale < 2e-6, k
        return
    # the probes decode FP16 values: re-encoding recovers them up to FP64 rounding of the shift
    g = stored_values(got, prm).astype(np.float16).astype(np.float64)
    w = stored_values(want, prm)
    w16 = w.astype(np.float16).astype(np.float64)
    for k in range(5):
        blk = slice(7 * k, 7 * k + 7)
        bound = spacing(w16[blk], storage) + 16 * 2.0 ** -24 * np.abs(w[blk]).max()
        assert np.all(np.abs(g[blk] - w16[blk]) <= bound), (k, float(np.max(np.abs(g[blk] - w16[blk]) / bound)))
    share = float((g != w16).mean())
    assert share < 2e-3, share


def test_capacity_moment_storage_sampled_cells():
    """1024^3 in FP32 as moments (two buffers of 20 values per cell: 172 GB, where FP32
    populations fit only at 768^3 with one buffer): after 5 sweeps, one more sweep of 2000
    sampled cells against the oracle's update of the probed pre-step populations, within 2e-6
    of each field's largest population.  Skipped if the device cannot hold it."""
    torch = pytest.importorskip("torch")
    n = 1024
    prm = inputs.tgv3d(n, nxyz=(1, 1, 1)).params.replace(nx=n, ny=n, nz=n, streaming=2)
    torch.cuda.empty_cache()
    capi.grlb_trim_pool()  # earlier tests' domains went back to the library's pool
    free, _ = torch.cuda.mem_get_info()
    if capi.grlb_bytes_for(prm) + 5 * 8 * n ** 3 + (2 << 30) > free:
        pytest.skip("device memory")
    d = capi.Domain(prm)
    _, rho, u, p = inputs.tgv3d_device(n)
    capi.grlb_init_primitive_device(d.h, rho.data_ptr(), u.data_ptr(), p.data_ptr())
    torch.cuda.synchronize()
    del rho, u, p
    torch.cuda.empty_cache()
    d.step(5)
    N = prm.ncells
    rng = np.random.default_rng(12)
    edges = [0, 1, n - 1, n, n * n - 1, n * n, N - n, N - 128, N - 1]
    cells = np.unique(np.concatenate([rng.integers(0, N, 2000), edges])).astype(np.int64)
    want, _ = oracle_update_cells(prm, lambda cs: capi.grlb_read_cells(d.h, cs), cells)
    d.step(1)
    got = capi.grlb_read_cells(d.h, cells)
    d.close()
    torch.cuda.empty_cache()
    for k in range(5):
        blk = slice(7 * k, 7 * k + 7)
        scale = max(np.abs(want[blk]).max(), 1e-12)
        assert np.abs(got[blk] - want[blk]).max() / scale < 2e-6, k
