"""GPU spectral post-processing (grlb_spectral_diag through the C ABI) against the FP64 oracle
and against closed forms.

Tolerances (FP32 populations, FP32 complex FFT): after n sweeps the CUDA and oracle states
agree to 1e-5 relative (the sweep parity bar); the spectrum and the dissipation sums are
quadratic in u, so energetic shells and eps_s agree to 1e-4 relative, with an absolute floor
of 1e-6 of the total energy for nearly empty shells and 1e-4 of the total dissipation for the
dilatational part.  At step 0 (fields rounded once to FP32) the bars are 1e-5.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import spectral
from paper_2609_16361_b300 import capi, inputs
from tests.common import run_oracle

pytestmark = pytest.mark.gpu


def gpu_domain(case, steps=0, streaming=0):
    prm = case.params.replace(streaming=streaming)
    d = capi.Domain(prm)
    d.init(case.rho, case.u, case.p)
    if steps:
        d.step(steps)
    return d


def assert_spectra_close(Eg, Eo, rel, floor):
    tot = Eo.sum()
    err = np.abs(Eg - Eo)
    assert np.all(err <= rel * np.abs(Eo) + floor * tot), (np.argmax(err - rel * np.abs(Eo)), err.max())


def assert_sums_close(sg, so, rel):
    assert sg["eps_s"] == pytest.approx(so["eps_s"], rel=rel)
    assert abs(sg["eps_d"] - so["eps_d"]) <= rel * (so["eps_s"] + so["eps_d"])
    assert sg["ke_u"] == pytest.approx(so["ke_u"], rel=rel)


@pytest.mark.parametrize("n", [16, 32, 256, 512])
def test_taylor_green_initial_closed_form(n):
    """All energy at |m| = sqrt 3 (shell 2): s^2/8 per cell; sum mu |curl u|^2 =
    N mu_L (s dx)^2 3/4; no divergence.  256^3 is the full benchmark size; lines of n <= 256
    points take the four-step kernels (n = 16: one thread per line), n = 512 the Stockham
    kernels."""
    c = inputs.tgv3d(n)
    d = gpu_domain(c)
    E, s = d.spectral()
    sL, dx = c.params.dt / c.params.dx, c.params.dx
    mu_L = c.params.mu_ref * c.params.dt / dx ** 2
    assert len(E) == spectral.shells(n, n, n)
    assert E[2] == pytest.approx(sL * sL / 8.0, rel=1e-5)
    assert np.delete(E, 2).sum() < 1e-6 * E[2]
    assert s["eps_s"] == pytest.approx(n ** 3 * mu_L * (sL * dx) ** 2 * 0.75, rel=1e-5)
    assert s["eps_d"] < 1e-6 * s["eps_s"]
    d.close()


@pytest.mark.parametrize("n,steps", [(32, 0), (32, 30), (16, 12), (128, 0)])
def test_random_smooth_parity(n, steps):
    c = inputs.random_smooth(n, n, n, seed=11)
    d = gpu_domain(c, steps)
    Eg, sg = d.spectral()
    o = run_oracle(c, steps)
    Eo, so = spectral.from_oracle(o)
    rel, floor = (1e-5, 1e-7) if steps == 0 else (1e-4, 1e-6)
    assert_spectra_close(Eg, Eo, rel, floor)
    assert_sums_close(sg, so, rel)
    d.close()


def test_taylor_green_64_after_steps():
    c = inputs.tgv3d(64, mach=1.25, re=100.0)
    d = gpu_domain(c, 40)
    Eg, sg = d.spectral()
    Eo, so = spectral.from_oracle(run_oracle(c, 40))
    assert_spectra_close(Eg, Eo, 1e-4, 1e-6)
    assert_sums_close(sg, so, 1e-4)
    d.close()


@pytest.mark.parametrize("n", [64, 32])
def test_square_2d_box(n):
    """n = 64: four-step x transforms; n = 32 (fewer rows than a four-step CTA takes): the
    Stockham kernels."""
    c = inputs.tgv2d(n)
    d = gpu_domain(c, 20)
    Eg, sg = d.spectral()
    Eo, so = spectral.from_oracle(run_oracle(c, 20))
    assert len(Eg) == spectral.shells(n, n, 1)
    assert_spectra_close(Eg, Eo, 1e-4, 1e-6)
    assert_sums_close(sg, so, 1e-4)
    d.close()


def test_one_buffer_layout_after_odd_step():
    """The one-buffer (AA) state after an odd step is read through the gather: same result
    as the two-buffer state after the same steps (FP32 rounding)."""
    c = inputs.random_smooth(32, 32, 32, seed=3)
    a = gpu_domain(c, 7, streaming=0)
    b = gpu_domain(c, 7, streaming=1)
    Ea, sa = a.spectral()
    Eb, sb = b.spectral()
    assert_spectra_close(Eb, Ea, 1e-5, 1e-7)
    assert_sums_close(sb, sa, 1e-5)
    a.close()
    b.close()


def test_f16_storage_close_to_oracle():
    c = inputs.random_smooth(32, 32, 32, seed=2, storage=inputs.STORE_F16)
    d = gpu_domain(c, 10)
    Eg, sg = d.spectral()
    Eo, so = spectral.from_oracle(run_oracle(c, 10))
    big = Eo > 1e-3 * Eo.sum()
    assert np.all(np.abs(Eg[big] / Eo[big] - 1.0) < 1e-2)
    assert sg["eps_s"] == pytest.approx(so["eps_s"], rel=2e-2)
    d.close()


def test_reproducible_and_partial_bins():
    c = inputs.random_smooth(32, 32, 32, seed=4)
    d = gpu_domain(c, 5)
    E1, s1 = d.spectral()
    E2, s2 = d.spectral()
    assert np.array_equal(E1, E2) and s1 == s2
    E3, s3 = capi.grlb_spectral_diag(d.h, 5)
    assert np.array_equal(E3, E1[:5]) and s3 == s1
    E4, _ = capi.grlb_spectral_diag(d.h, len(E1) + 4)
    assert np.array_equal(E4[:len(E1)], E1) and not E4[len(E1):].any()
    d.close()


def test_rejects_unsupported_domains():
    sod = gpu_domain(inputs.sod(64))
    with pytest.raises(capi.GrlbError) as e:
        sod.spectral(8)
    assert e.value.status == -1  # GRLB_EINVAL
    sod.close()
    odd = gpu_domain(inputs.random_smooth(24, 24, 24, seed=1))
    with pytest.raises(capi.GrlbError):
        odd.spectral(8)
    odd.close()


def test_ffma_probe_runs_and_leaves_sink():
    import torch
    sink = torch.zeros(148 * 256, device="cuda")
    st = torch.cuda.current_stream()
    n = capi.grlb_ffma_probe(148, 16, sink.data_ptr(), st.cuda_stream)
    torch.cuda.synchronize()
    assert n == 148 * 8 * 16 * 128
    assert not sink.any()
