"""Failure paths on the GPU, made to happen without faulting or hanging it.

* A bounded device-side wait that nothing completes gives up after its limit
  and is reported (dmrt_probe_bounded_wait runs the step kernels' wait routine
  on an mbarrier nothing arrives on); the GPU and later steps are unaffected.
* A non-finite state is reported as DMRT_E_DIVERGED (tests/test_cuda_parity.py),
  and a long dmrt_step call stops at its next poll of the error word instead
  of stepping a diverged state to the end.
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


def test_long_step_call_stops_at_the_divergence_poll(D):
    # A NaN temperature in one node: dmrt_step polls the error word each time the
    # step count passes a multiple of 65536 and returns DMRT_E_DIVERGED there.
    cav = inputs.Cavity(16, 16, 1e4, 0.01, noise_amp=1e-3, seed=6)
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=64)
    st = sim.get_state()
    st[9, 5, 7] = np.nan
    sim.set_state(st)
    want = 3 * 65536 + 100
    with pytest.raises(D.DmrtError) as ei:
        sim.step(want)
    assert ei.value.code == D.DMRT_E_DIVERGED
    assert sim.steps_done == 65536
    sim.close()
    # A healthy run of the same length is not interrupted (Ra 1e3, Pr 1: stable
    # on this small grid for any number of steps).
    ok = D.Cavity2D.from_inputs(inputs.Cavity(16, 16, 1e3, 1.0, noise_amp=1e-3, seed=6), nu_capacity=64)
    ok.step(want)
    ok.check()
    assert ok.steps_done == want
    ok.close()
