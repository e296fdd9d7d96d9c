"""Failure paths on the GPU, made to happen without faulting or hanging it.

* A bounded device-side wait that nothing completes gives up after its limit
  and is reported (dmrt_probe_bounded_wait runs the step kernels' wait routine
  on an mbarrier nothing arrives on); the GPU and later steps are unaffected.
* A non-finite state is reported as DMRT_E_DIVERGED (tests/test_cuda_parity.py).
"""
import ctypes

import numpy as np
import pytest

from paper_1601_04633_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1601_04633_gb300 import dmrt

    return dmrt


def test_bounded_wait_gives_up_and_the_context_stays_usable(D):
    import torch

    L = D.load()
    stream = torch.cuda.current_stream().cuda_stream
    cav = inputs.Cavity(600, 40, 1e5, 0.01, noise_amp=1e-3, seed=5)
    ref = D.Cavity2D.from_inputs(cav, nu_capacity=64)
    ref.step(20)
    ref.check()
    waited = ctypes.c_int64(0)
    for limit_ms in (5, 50):
        rc = L.dmrt_probe_bounded_wait(limit_ms * 1_000_000, ctypes.c_void_p(stream), ctypes.byref(waited))
        assert rc == D.DMRT_E_TIMEOUT
        assert limit_ms * 1e6 <= waited.value < limit_ms * 1e6 + 2e8
    # Stepping after the expired wait gives the same bits as before it.
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=64)
    sim.step(20)
    sim.check()
    assert np.array_equal(sim.get_state(), ref.get_state())
    sim.close()
    ref.close()
    assert L.dmrt_probe_bounded_wait(10, ctypes.c_void_p(stream), None) == D.DMRT_E_ARG
