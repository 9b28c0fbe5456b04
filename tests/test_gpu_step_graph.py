"""grlb_step replays the sweeps of small domains from a CUDA graph (on a non-default stream):
the states it produces are bitwise those of one launch per step, from either buffer / step
parity, for two-buffer and one-buffer streaming, and after the source term is replaced."""
import numpy as np
import pytest

from paper_2609_16361_b300 import capi, inputs

pytestmark = pytest.mark.gpu


def pair(case, stream, streaming=0):
    prm = case.params.replace(streaming=streaming)
    a = capi.Domain(prm, stream=stream.cuda_stream)  # multi-step calls: graph replay
    b = capi.Domain(prm, stream=stream.cuda_stream)  # single steps: plain launches
    for d in (a, b):
        d.init(case.rho, case.u, case.p)
    return a, b


def single_steps(d, n):
    for _ in range(n):
        d.step(1)


@pytest.mark.parametrize("streaming", [0, 1])
@pytest.mark.parametrize("case", [lambda: inputs.sod(400), lambda: inputs.becker(512, 3.0, ny=4, nz=4),
                                  lambda: inputs.random_smooth(40, 21, 7, seed=3)])
def test_graph_replay_is_bitwise_one_launch_per_step(case, streaming):
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    c = case()
    a, b = pair(c, stream, streaming)
    a.step(37)            # odd count: graph replays plus plain sweeps
    single_steps(b, 37)
    a.step(1)
    single_steps(b, 1)
    a.step(50)            # starts at the other parity: one plain sweep aligns it
    single_steps(b, 50)
    assert a.steps == b.steps == 88
    stream.synchronize()
    assert np.array_equal(capi.grlb_save(a.h), capi.grlb_save(b.h))
    assert np.array_equal(a.conserved(), b.conserved())
    a.close()
    b.close()


def test_replacing_the_source_drops_the_graph():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    c = inputs.random_smooth(24, 20, 16, seed=5, collision=inputs.COLL_BGK)
    a, b = pair(c, stream)
    S1 = torch.full((5, c.params.ncells), 1e-6, dtype=torch.float32, device="cuda")
    S2 = torch.full((5, c.params.ncells), -2e-6, dtype=torch.float32, device="cuda")
    for S in (S1, S2, None):
        for d in (a, b):
            capi.grlb_set_source_device(d.h, None if S is None else S.data_ptr())
        a.step(20)
        single_steps(b, 20)
    stream.synchronize()
    assert np.array_equal(capi.grlb_save(a.h), capi.grlb_save(b.h))
    a.close()
    b.close()
